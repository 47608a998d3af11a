// Vector kernels: interface pack/unpack, link compression, the two deflation
// passes of Eq. 3 (projection coefficients c_i = phi_i^dagger psi, then
// psi_perp = psi - sum c_i phi_i together with the correction
// sum sgn(lambda_i) c_i phi_i), and the BLAS-1 steps of CG with FP64 global
// sums.  Every reduction runs on a fixed grid of kReduceBlocks x
// kReduceThreads with a fixed summation order, so results are bitwise
// reproducible run to run.
#include "common.cuh"
#include "internal.h"

namespace ov {

constexpr int kThreads = 256;

static inline unsigned grid_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// block reduction of a double2 (all threads of the block participate)

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Returns the block sum in thread 0.
__device__ __forceinline__ double2 block_sum(double2 v, double2* smem /* >= 32 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) smem[wid] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    r = (lane < nw) ? smem[lane] : make_double2(0.0, 0.0);
    r = warp_sum(r);
  }
  return r;
}

// arithmetic type of an operation touching storages A and B
template <class A, class B> struct Arith { using R = float; };
template <> struct Arith<F64, F64> { using R = double; };
template <class B> struct Arith<F64, B> { using R = double; };
template <class A> struct Arith<A, F64> { using R = double; };

// dispatch helpers --------------------------------------------------------
#define OV_DISPATCH1(p, T, ...)                  \
  switch (p) {                                   \
    case OP_F64: { using T = F64; __VA_ARGS__; } break; \
    case OP_F32: { using T = F32; __VA_ARGS__; } break; \
    case OP_F16: { using T = F16; __VA_ARGS__; } break; \
    case OP_B16: { using T = B16; __VA_ARGS__; } break; \
  }

// ---------------------------------------------------------------------------
// interface <-> internal

template <class T, class IR>
__global__ void k_pack_spinor(const IR* __restrict__ in, char* __restrict__ out, int64_t V, int64_t rhs_bytes,
                              double scale, int g5) {
  using R = typename Arith<T, T>::R;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int rhs = blockIdx.y;
  const IR* p = in + ((int64_t)rhs * V + s) * 24;
  Spinor<R> o;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const R sg = (g5 && k >= 6) ? R(-scale) : R(scale);
    o.c[k] = {sg * R(p[2 * k]), sg * R(p[2 * k + 1])};
  }
  store_spinor_as<T, R>(out + rhs * rhs_bytes, s, V, o);
}

template <class T, class IR>
__global__ void k_unpack_spinor(const char* __restrict__ in, IR* __restrict__ out, int64_t V, int64_t rhs_bytes,
                                double scale) {
  using R = typename Arith<T, T>::R;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int rhs = blockIdx.y;
  Spinor<R> o;
  load_spinor_as<T, R>(in + rhs * rhs_bytes, s, V, o);
  IR* p = out + ((int64_t)rhs * V + s) * 24;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    p[2 * k] = IR(R(scale) * o.c[k].re);
    p[2 * k + 1] = IR(R(scale) * o.c[k].im);
  }
}

void launch_pack_spinor(OpPrec p, IfaceType it, const LatticeH& g, const void* in, void* out, int nrhs,
                        double scale, int g5, cudaStream_t st) {
  const int64_t rb = (int64_t)spinor_bytes_per_site(p) * g.V;
  dim3 grid(grid_for(g.V), nrhs);
  OV_DISPATCH1(p, T, {
    if (it == IF_C128)
      k_pack_spinor<T, double><<<grid, kThreads, 0, st>>>(static_cast<const double*>(in), static_cast<char*>(out),
                                                          g.V, rb, scale, g5);
    else
      k_pack_spinor<T, float><<<grid, kThreads, 0, st>>>(static_cast<const float*>(in), static_cast<char*>(out),
                                                         g.V, rb, scale, g5);
  });
}

void launch_unpack_spinor(OpPrec p, IfaceType it, const LatticeH& g, const void* in, void* out, int nrhs,
                          double scale, cudaStream_t st) {
  const int64_t rb = (int64_t)spinor_bytes_per_site(p) * g.V;
  dim3 grid(grid_for(g.V), nrhs);
  OV_DISPATCH1(p, T, {
    if (it == IF_C128)
      k_unpack_spinor<T, double><<<grid, kThreads, 0, st>>>(static_cast<const char*>(in), static_cast<double*>(out),
                                                            g.V, rb, scale);
    else
      k_unpack_spinor<T, float><<<grid, kThreads, 0, st>>>(static_cast<const char*>(in), static_cast<float*>(out),
                                                           g.V, rb, scale);
  });
}

template <class T, int LREC>
__global__ void k_pack_links(const double2* __restrict__ in, void* __restrict__ out, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int mu = blockIdx.y;
  const double2* u = in + ((int64_t)mu * V + s) * 9;
  if constexpr (std::is_same<T, F64>::value) {
    double2* q = static_cast<double2*>(out) + (int64_t)mu * 9 * V;
#pragma unroll
    for (int e = 0; e < 9; ++e) q[e * V + s] = u[e];
  } else if constexpr (std::is_same<T, F32>::value) {
    float4* q = static_cast<float4*>(out) + (int64_t)mu * 3 * V;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      q[c * V + s] = make_float4((float)u[2 * c].x, (float)u[2 * c].y, (float)u[2 * c + 1].x, (float)u[2 * c + 1].y);
  } else if constexpr (LREC == 18) {  // entries 0-3, 4-7 as uint4 chunks, entry 8 as one word
    uint32_t w[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) w[e] = pack2<T>((float)u[e].x, (float)u[e].y);
    uint4* q = static_cast<uint4*>(out);
    q[(int64_t)mu * V + s] = make_uint4(w[0], w[1], w[2], w[3]);
    q[(int64_t)(4 + mu) * V + s] = make_uint4(w[4], w[5], w[6], w[7]);
    reinterpret_cast<uint32_t*>(q + (int64_t)8 * V)[(int64_t)mu * V + s] = w[8];
  } else {
    uint2* q = static_cast<uint2*>(out) + (int64_t)mu * 3 * V;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 v;
      v.x = pack2<T>((float)u[2 * c].x, (float)u[2 * c].y);
      v.y = pack2<T>((float)u[2 * c + 1].x, (float)u[2 * c + 1].y);
      q[c * V + s] = v;
    }
  }
}

// FP64 packed links (all 9 entries, [(mu * 9 + e) V + s]) back to the
// interface layout complex128 [4][V][3][3].
__global__ void k_unpack_links_f64(const double2* __restrict__ in, double2* __restrict__ out, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int mu = blockIdx.y;
  const double2* q = in + (int64_t)mu * 9 * V;
  double2* u = out + ((int64_t)mu * V + s) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) u[e] = q[(int64_t)e * V + s];
}

void launch_unpack_links_f64(const LatticeH& g, const void* packed, void* out, cudaStream_t st) {
  dim3 grid(grid_for(g.V), 4);
  k_unpack_links_f64<<<grid, kThreads, 0, st>>>(static_cast<const double2*>(packed), static_cast<double2*>(out),
                                                 (int)g.V);
}

void launch_pack_links(OpPrec p, int lrec, const LatticeH& g, const void* in, void* out, cudaStream_t st) {
  dim3 grid(grid_for(g.V), 4);
  const double2* src = static_cast<const double2*>(in);
  const int V = (int)g.V;
  switch (p) {
    case OP_F64: k_pack_links<F64, 18><<<grid, kThreads, 0, st>>>(src, out, V); break;
    case OP_F32: k_pack_links<F32, 12><<<grid, kThreads, 0, st>>>(src, out, V); break;
    case OP_F16:
      if (lrec == 18) k_pack_links<F16, 18><<<grid, kThreads, 0, st>>>(src, out, V);
      else k_pack_links<F16, 12><<<grid, kThreads, 0, st>>>(src, out, V);
      break;
    case OP_B16:
      if (lrec == 18) k_pack_links<B16, 18><<<grid, kThreads, 0, st>>>(src, out, V);
      else k_pack_links<B16, 12><<<grid, kThreads, 0, st>>>(src, out, V);
      break;
  }
}

// ---------------------------------------------------------------------------
// deflation

constexpr int kDeflChunk = 8;  // eigenvectors per pass over psi

template <class TE, class TS>
__global__ void __launch_bounds__(kReduceThreads) k_defl_dot(const char* __restrict__ evecs, int n_ev,
                                                             const char* __restrict__ psi, int64_t V, int g5,
                                                             double2* __restrict__ partial) {
  using R = typename Arith<TE, TS>::R;
  __shared__ double2 smem[32];
  const int64_t evec_bytes = (int64_t)Store<TE>::bytes_per_site * V;
  for (int i0 = 0; i0 < n_ev; i0 += kDeflChunk) {
    // a thread's few sites (V / (grid x block), ~4 at 24^3 x 48) are summed in
    // the arithmetic type and converted to FP64 once, so that FP32 vectors keep
    // the slow FP64 pipe out of the site loop (for FP64 the sum is unchanged)
    cplx<R> acc[kDeflChunk];
#pragma unroll
    for (int j = 0; j < kDeflChunk; ++j) acc[j] = {R(0), R(0)};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
      Spinor<R> x;
      load_spinor_as<TS, R>(psi, s, V, x);
      if (g5) {
#pragma unroll
        for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
      }
#pragma unroll
      for (int j = 0; j < kDeflChunk; ++j) {
        if (i0 + j < n_ev) {
          Spinor<R> f;
          load_spinor_as<TE, R>(evecs + (i0 + j) * evec_bytes, s, V, f);
          cplx<R> d = {R(0), R(0)};
#pragma unroll
          for (int k = 0; k < 12; ++k) d = d + cmulc(f.c[k], x.c[k]);
          acc[j] = acc[j] + d;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kDeflChunk; ++j) {
      if (i0 + j < n_ev) {
        double2 r = block_sum(make_double2((double)acc[j].re, (double)acc[j].im), smem);
        if (threadIdx.x == 0) partial[(int64_t)(i0 + j) * gridDim.x + blockIdx.x] = r;
      }
    }
  }
}

void launch_defl_dot(OpPrec pv, const LatticeH& g, const void* evecs, int n_ev, const void* psi, int g5,
                     double2* partial, cudaStream_t st) {
  if (n_ev <= 0) return;
  OV_DISPATCH1(pv, T, {
    k_defl_dot<T, T><<<kReduceBlocks, kReduceThreads, 0, st>>>(static_cast<const char*>(evecs), n_ev,
                                                               static_cast<const char*>(psi), g.V, g5, partial);
  });
}

__global__ void k_reduce_partials(const double2* __restrict__ partial, int nblk, double2* __restrict__ out) {
  __shared__ double2 smem[32];
  const int i = blockIdx.x;
  double2 v = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double2 p = partial[(int64_t)i * nblk + b];
    v.x += p.x;
    v.y += p.y;
  }
  v = block_sum(v, smem);
  if (threadIdx.x == 0) out[i] = v;
}

void launch_reduce_partials(const double2* partial, int n, int nblk, double2* out, cudaStream_t st) {
  if (n <= 0) return;
  k_reduce_partials<<<n, 256, 0, st>>>(partial, nblk, out);
}

// TV: storage of phi_i, psi and d; TP: storage of psi_perp.
template <class TV, class TP>
__global__ void k_defl_combine(const char* __restrict__ evecs, int n_ev, const double2* __restrict__ c,
                               int cstride, const double* __restrict__ sgn, const char* __restrict__ psi, int64_t V, int g5,
                               double scale, char* __restrict__ psi_perp, char* __restrict__ d) {
  using R = typename Arith<TV, TV>::R;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int64_t evec_bytes = (int64_t)Store<TV>::bytes_per_site * V;
  Spinor<R> x, corr;
  load_spinor_as<TV, R>(psi, s, V, x);
  if (g5) {
#pragma unroll
    for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) corr.c[k] = {R(0), R(0)};
  for (int i = 0; i < n_ev; ++i) {
    Spinor<R> f;
    load_spinor_as<TV, R>(evecs + i * evec_bytes, s, V, f);
    const double2 cd = c[(int64_t)i * cstride];
    const cplx<R> ci = {R(cd.x), R(cd.y)};
    const R si = R(sgn[i]);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cplx<R> t = cmul(ci, f.c[k]);
      x.c[k] = x.c[k] - t;
      corr.c[k] = corr.c[k] + si * t;
    }
  }
  const R sc = R(scale);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    x.c[k] = sc * x.c[k];
    corr.c[k] = sc * corr.c[k];
  }
  store_spinor_as<TP, R>(psi_perp, s, V, x);
  if (d != nullptr) store_spinor_as<TV, R>(d, s, V, corr);
}

void launch_defl_combine(OpPrec pv, OpPrec pp, const LatticeH& g, const void* evecs, int n_ev, const double2* c,
                         int cstride, const double* sgn, const void* psi, int g5, double scale, void* psi_perp, void* d,
                         cudaStream_t st) {
  const char* e = static_cast<const char*>(evecs);
  const char* x = static_cast<const char*>(psi);
  char* pp_ = static_cast<char*>(psi_perp);
  char* dd = static_cast<char*>(d);
  const unsigned gr = grid_for(g.V);
  if (pv == OP_F64) {
    k_defl_combine<F64, F64><<<gr, kThreads, 0, st>>>(e, n_ev, c, cstride, sgn, x, g.V, g5, scale, pp_, dd);
  } else {
    OV_DISPATCH1(pp, TP, {
      k_defl_combine<F32, TP><<<gr, kThreads, 0, st>>>(e, n_ev, c, cstride, sgn, x, g.V, g5, scale, pp_, dd);
    });
  }
}

// Several right-hand sides at once (FP32 vectors): thread = (site, float4
// chunk c = complex 2c, 2c+1), RHS tile of kCombineRB in registers, so each
// eigenvector chunk is read once per tile instead of once per right-hand side.
// c[i*cstride_i + r] holds c_i for right-hand side r (the batched projection).
template <class TP, int kCombineRB>
__global__ void __launch_bounds__(256) k_defl_combine_multi(const float4* __restrict__ evecs, int n_ev,
                                                            const double2* __restrict__ c, int nrhs,
                                                            const double* __restrict__ sgn,
                                                            const float4* __restrict__ psi, int V, int g5,
                                                            float scale, char* __restrict__ psi_perp,
                                                            float4* __restrict__ d) {
  __shared__ float2 cs[128 * kCombineRB];
  __shared__ float ss[128];
  const int r0 = blockIdx.y * kCombineRB;
  const int nv = min(kCombineRB, nrhs - r0);
  for (int idx = threadIdx.x; idx < n_ev * kCombineRB; idx += blockDim.x) {
    const int i = idx / kCombineRB, r = idx % kCombineRB;
    const double2 v = (r < nv) ? c[(int64_t)i * nrhs + r0 + r] : make_double2(0.0, 0.0);
    cs[idx] = make_float2((float)v.x, (float)v.y);
  }
  for (int i = threadIdx.x; i < n_ev; i += blockDim.x) ss[i] = (float)sgn[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int ch = blockIdx.z;  // float4 chunk 0..5
  const int64_t off = (int64_t)ch * V + s;
  const float gs = (g5 && ch >= 3) ? -1.f : 1.f;  // chunks 3..5 hold spins 2, 3
  float4 x[kCombineRB], corr[kCombineRB];
#pragma unroll
  for (int r = 0; r < kCombineRB; ++r) {
    x[r] = corr[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < nv) {
      const float4 v = __ldg(psi + (int64_t)(r0 + r) * 6 * V + off);
      x[r] = make_float4(gs * v.x, gs * v.y, gs * v.z, gs * v.w);
    }
  }
  for (int i = 0; i < n_ev; ++i) {
    const float4 f = __ldg(evecs + (int64_t)i * 6 * V + off);
    const float si = ss[i];
#pragma unroll
    for (int r = 0; r < kCombineRB; ++r) {
      const float2 ci = cs[i * kCombineRB + r];
      const float t0r = ci.x * f.x - ci.y * f.y, t0i = ci.x * f.y + ci.y * f.x;
      const float t1r = ci.x * f.z - ci.y * f.w, t1i = ci.x * f.w + ci.y * f.z;
      x[r].x -= t0r;
      x[r].y -= t0i;
      x[r].z -= t1r;
      x[r].w -= t1i;
      corr[r].x += si * t0r;
      corr[r].y += si * t0i;
      corr[r].z += si * t1r;
      corr[r].w += si * t1i;
    }
  }
#pragma unroll
  for (int r = 0; r < kCombineRB; ++r) {
    if (r >= nv) break;
    const float4 xo = make_float4(scale * x[r].x, scale * x[r].y, scale * x[r].z, scale * x[r].w);
    d[(int64_t)(r0 + r) * 6 * V + off] =
        make_float4(scale * corr[r].x, scale * corr[r].y, scale * corr[r].z, scale * corr[r].w);
    if constexpr (std::is_same<TP, F32>::value) {
      reinterpret_cast<float4*>(psi_perp)[(int64_t)(r0 + r) * 6 * V + off] = xo;
    } else {
      // 16-bit chunk ch/2 holds complex 4*(ch/2) .. +3; this thread's two are its half ch%2
      uint2 w;
      w.x = pack2<TP>(xo.x, xo.y);
      w.y = pack2<TP>(xo.z, xo.w);
      uint2* q = reinterpret_cast<uint2*>(psi_perp + (int64_t)(r0 + r) * 48 * V);
      q[((int64_t)(ch >> 1) * V + s) * 2 + (ch & 1)] = w;
    }
  }
}

template <int RB>
static void combine_multi_rb(OpPrec pp, const LatticeH& g, const void* evecs, int n_ev, const double2* c, int nrhs,
                             const double* sgn, const void* psi, int g5, double scale, void* psi_perp, void* d,
                             cudaStream_t st) {
  dim3 grid(grid_for(g.V), (nrhs + RB - 1) / RB, 6);
  const float4* e = static_cast<const float4*>(evecs);
  const float4* x = static_cast<const float4*>(psi);
  char* pp_ = static_cast<char*>(psi_perp);
  float4* dd = static_cast<float4*>(d);
  switch (pp) {
    case OP_F32:
      k_defl_combine_multi<F32, RB><<<grid, kThreads, 0, st>>>(e, n_ev, c, nrhs, sgn, x, (int)g.V, g5, (float)scale, pp_, dd);
      break;
    case OP_F16:
      k_defl_combine_multi<F16, RB><<<grid, kThreads, 0, st>>>(e, n_ev, c, nrhs, sgn, x, (int)g.V, g5, (float)scale, pp_, dd);
      break;
    case OP_B16:
      k_defl_combine_multi<B16, RB><<<grid, kThreads, 0, st>>>(e, n_ev, c, nrhs, sgn, x, (int)g.V, g5, (float)scale, pp_, dd);
      break;
    default:
      break;
  }
}

void launch_defl_combine_multi(OpPrec pp, const LatticeH& g, const void* evecs, int n_ev, const double2* c, int nrhs,
                               const double* sgn, const void* psi, int g5, double scale, void* psi_perp, void* d,
                               cudaStream_t st) {
  // right-hand sides per thread: each tile re-reads every eigenvector, so one
  // tile of up to 12 (12 point sources at 24^3 x 48, 40 eigenvectors: 1.80 ms
  // against 2.02 ms for tiles of 6 and 2.12 ms for tiles of 4)
  if (nrhs > 6) combine_multi_rb<12>(pp, g, evecs, n_ev, c, nrhs, sgn, psi, g5, scale, psi_perp, d, st);
  else if (nrhs > 4) combine_multi_rb<6>(pp, g, evecs, n_ev, c, nrhs, sgn, psi, g5, scale, psi_perp, d, st);
  else combine_multi_rb<4>(pp, g, evecs, n_ev, c, nrhs, sgn, psi, g5, scale, psi_perp, d, st);
}

// ---------------------------------------------------------------------------
// BLAS-1 on same-storage vectors, treated as flat arrays of complex numbers
// (layout-agnostic: all operands share the layout).  A "unit" is one storage
// chunk; unit_complex complex numbers per unit.

template <class T> struct Unit;
template <> struct Unit<F64> {
  using U = double2;
  static constexpr int n = 1;
  __device__ static void load(const U& u, cplx<double>* c) { c[0] = {u.x, u.y}; }
  __device__ static U store(const cplx<double>* c) { return make_double2(c[0].re, c[0].im); }
};
template <> struct Unit<F32> {
  using U = float4;
  static constexpr int n = 2;
  __device__ static void load(const U& u, cplx<float>* c) {
    c[0] = {u.x, u.y};
    c[1] = {u.z, u.w};
  }
  __device__ static U store(const cplx<float>* c) { return make_float4(c[0].re, c[0].im, c[1].re, c[1].im); }
};
template <class T> struct Unit16 {
  using U = uint4;
  static constexpr int n = 4;
  __device__ static void load(const U& u, cplx<float>* c) {
    float2 a = unpack2<T>(u.x), b = unpack2<T>(u.y), d = unpack2<T>(u.z), e = unpack2<T>(u.w);
    c[0] = {a.x, a.y};
    c[1] = {b.x, b.y};
    c[2] = {d.x, d.y};
    c[3] = {e.x, e.y};
  }
  __device__ static U store(const cplx<float>* c) {
    U u;
    u.x = pack2<T>(c[0].re, c[0].im);
    u.y = pack2<T>(c[1].re, c[1].im);
    u.z = pack2<T>(c[2].re, c[2].im);
    u.w = pack2<T>(c[3].re, c[3].im);
    return u;
  }
};
template <> struct Unit<F16> : Unit16<F16> {};
template <> struct Unit<B16> : Unit16<B16> {};

template <class T>
static inline int64_t n_units(int64_t V, int nrhs) {
  return V * nrhs * 12 / Unit<T>::n;
}

template <class T>
__global__ void __launch_bounds__(kReduceThreads) k_dot_partial(const typename Unit<T>::U* __restrict__ a,
                                                                const typename Unit<T>::U* __restrict__ b, int64_t n,
                                                                double2* __restrict__ partial, int norm_only) {
  using R = typename Arith<T, T>::R;
  constexpr int m = Unit<T>::n;
  __shared__ double2 smem[32];
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx<R> x[m], y[m];
    Unit<T>::load(a[i], x);
    if (norm_only) {
      R t = R(0);
#pragma unroll
      for (int k = 0; k < m; ++k) t += x[k].re * x[k].re + x[k].im * x[k].im;
      acc.x += (double)t;
    } else {
      Unit<T>::load(b[i], y);
      cplx<R> t = {R(0), R(0)};
#pragma unroll
      for (int k = 0; k < m; ++k) t = t + cmulc(x[k], y[k]);
      acc.x += (double)t.re;
      acc.y += (double)t.im;
    }
  }
  acc = block_sum(acc, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

void launch_dot_partial(OpPrec p, const void* a, const void* b, int64_t V, int nrhs, double2* partial,
                        cudaStream_t st) {
  OV_DISPATCH1(p, T, {
    using U = typename Unit<T>::U;
    k_dot_partial<T><<<kReduceBlocks, kReduceThreads, 0, st>>>(static_cast<const U*>(a), static_cast<const U*>(b),
                                                               n_units<T>(V, nrhs), partial, 0);
  });
}

void launch_norm2_partial(OpPrec p, const void* a, int64_t V, int nrhs, double2* partial, cudaStream_t st) {
  OV_DISPATCH1(p, T, {
    using U = typename Unit<T>::U;
    k_dot_partial<T><<<kReduceBlocks, kReduceThreads, 0, st>>>(static_cast<const U*>(a), static_cast<const U*>(a),
                                                               n_units<T>(V, nrhs), partial, 1);
  });
}

template <class T>
__global__ void __launch_bounds__(kReduceThreads) k_cg_update_xr(typename Unit<T>::U* __restrict__ x,
                                                                 typename Unit<T>::U* __restrict__ r,
                                                                 const typename Unit<T>::U* __restrict__ p,
                                                                 const typename Unit<T>::U* __restrict__ q,
                                                                 double alpha, int64_t n,
                                                                 double2* __restrict__ partial) {
  using R = typename Arith<T, T>::R;
  constexpr int m = Unit<T>::n;
  __shared__ double2 smem[32];
  const R al = R(alpha);
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx<R> xv[m], rv[m], pv[m], qv[m];
    Unit<T>::load(x[i], xv);
    Unit<T>::load(r[i], rv);
    Unit<T>::load(p[i], pv);
    Unit<T>::load(q[i], qv);
    R t = R(0);
#pragma unroll
    for (int k = 0; k < m; ++k) {
      xv[k] = xv[k] + al * pv[k];
      rv[k] = rv[k] - al * qv[k];
      t += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
    }
    x[i] = Unit<T>::store(xv);
    r[i] = Unit<T>::store(rv);
    acc.x += (double)t;
  }
  acc = block_sum(acc, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

void launch_cg_update_xr(OpPrec p, void* x, void* r, const void* pv, const void* q, double alpha, int64_t V, int nrhs,
                         double2* partial, cudaStream_t st) {
  OV_DISPATCH1(p, T, {
    using U = typename Unit<T>::U;
    k_cg_update_xr<T><<<kReduceBlocks, kReduceThreads, 0, st>>>(static_cast<U*>(x), static_cast<U*>(r),
                                                                static_cast<const U*>(pv), static_cast<const U*>(q),
                                                                alpha, n_units<T>(V, nrhs), partial);
  });
}

template <class T>
__global__ void k_axpby(double a, const typename Unit<T>::U* x, double b, const typename Unit<T>::U* y,
                        typename Unit<T>::U* out, int64_t n) {
  using R = typename Arith<T, T>::R;
  constexpr int m = Unit<T>::n;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  cplx<R> xv[m], yv[m];
  Unit<T>::load(x[i], xv);
  if (y != nullptr) {
    Unit<T>::load(y[i], yv);
#pragma unroll
    for (int k = 0; k < m; ++k) xv[k] = R(a) * xv[k] + R(b) * yv[k];
  } else {
#pragma unroll
    for (int k = 0; k < m; ++k) xv[k] = R(a) * xv[k];
  }
  out[i] = Unit<T>::store(xv);
}

void launch_axpby(OpPrec p, double a, const void* x, double b, const void* y, void* out, int64_t V, int nrhs,
                  cudaStream_t st) {
  OV_DISPATCH1(p, T, {
    using U = typename Unit<T>::U;
    const int64_t n = n_units<T>(V, nrhs);
    k_axpby<T><<<grid_for(n), kThreads, 0, st>>>(a, static_cast<const U*>(x), b, static_cast<const U*>(y),
                                                 static_cast<U*>(out), n);
  });
}

void launch_cg_update_p(OpPrec p, void* pv, const void* r, double beta, int64_t V, int nrhs, cudaStream_t st) {
  launch_axpby(p, 1.0, r, beta, pv, pv, V, nrhs, st);
}

// y = y + a x, complex a (GCR updates and orthogonalisation)
template <class T>
__global__ void k_caxpy(double2 a, const typename Unit<T>::U* __restrict__ x, typename Unit<T>::U* __restrict__ y,
                        int64_t n) {
  using R = typename Arith<T, T>::R;
  constexpr int m = Unit<T>::n;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cplx<R> ac = {R(a.x), R(a.y)};
  cplx<R> xv[m], yv[m];
  Unit<T>::load(x[i], xv);
  Unit<T>::load(y[i], yv);
#pragma unroll
  for (int k = 0; k < m; ++k) yv[k] = yv[k] + cmul(ac, xv[k]);
  y[i] = Unit<T>::store(yv);
}

void launch_caxpy(OpPrec p, double2 a, const void* x, void* y, int64_t V, int nrhs, cudaStream_t st) {
  OV_DISPATCH1(p, T, {
    using U = typename Unit<T>::U;
    const int64_t n = n_units<T>(V, nrhs);
    k_caxpy<T><<<grid_for(n), kThreads, 0, st>>>(a, static_cast<const U*>(x), static_cast<U*>(y), n);
  });
}

// One SUMR step on lazily normalised vectors (see SumrCoef): the deferred
// X term, the divided-difference pair, the new Krylov pair, and the squared
// norms of the new (unnormalised) Krylov pair in partial[] (x: V, y: T).
template <class T>
__global__ void __launch_bounds__(kReduceThreads) k_sumr_update(typename Unit<T>::U* __restrict__ v,
                                                                typename Unit<T>::U* __restrict__ vt,
                                                                const typename Unit<T>::U* __restrict__ w,
                                                                typename Unit<T>::U* __restrict__ dh,
                                                                typename Unit<T>::U* __restrict__ dth,
                                                                typename Unit<T>::U* __restrict__ x, SumrCoef c,
                                                                int64_t n, double2* __restrict__ partial) {
  using R = typename Arith<T, T>::R;
  constexpr int m = Unit<T>::n;
  __shared__ double2 smem[32];
  const cplx<R> cx = {R(c.cx.x), R(c.cx.y)}, mt = {R(c.mt.x), R(c.mt.y)}, mc = {R(c.mc.x), R(c.mc.y)},
                mcv = {R(c.mcv.x), R(c.mcv.y)};
  const R av = R(c.av), at = R(c.at), zv = R(c.zv);
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx<R> vv[m], tv[m], wv[m], dv[m], dtv[m], xv[m];
    Unit<T>::load(v[i], vv);
    Unit<T>::load(vt[i], tv);
    Unit<T>::load(w[i], wv);
    Unit<T>::load(dh[i], dv);
    Unit<T>::load(dth[i], dtv);
    Unit<T>::load(x[i], xv);
    R nv = R(0), nt = R(0);
#pragma unroll
    for (int k = 0; k < m; ++k) {
      xv[k] = xv[k] + cmul(cx, dv[k]);
      const cplx<R> t = av * vv[k] + zv * dv[k];
      dv[k] = t - cmul(mt, dtv[k]);
      dtv[k] = at * dtv[k] - cmul(mc, t);
      vv[k] = av * wv[k] - cmul(mt, tv[k]);
      tv[k] = at * tv[k] - cmul(mcv, wv[k]);
      nv += vv[k].re * vv[k].re + vv[k].im * vv[k].im;
      nt += tv[k].re * tv[k].re + tv[k].im * tv[k].im;
    }
    v[i] = Unit<T>::store(vv);
    vt[i] = Unit<T>::store(tv);
    dh[i] = Unit<T>::store(dv);
    dth[i] = Unit<T>::store(dtv);
    x[i] = Unit<T>::store(xv);
    acc.x += (double)nv;
    acc.y += (double)nt;
  }
  acc = block_sum(acc, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

void launch_sumr_update(OpPrec p, void* v, void* vt, const void* w, void* dh, void* dth, void* x, const SumrCoef& c,
                        int64_t V, double2* partial, cudaStream_t st) {
  OV_DISPATCH1(p, T, {
    using U = typename Unit<T>::U;
    k_sumr_update<T><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        static_cast<U*>(v), static_cast<U*>(vt), static_cast<const U*>(w), static_cast<U*>(dh), static_cast<U*>(dth),
        static_cast<U*>(x), c, n_units<T>(V, 1), partial);
  });
}

// per-site conversion between storages (layouts differ between storages)
template <class TI, class TO>
__global__ void k_convert(const char* __restrict__ in, char* out, int64_t V, int64_t in_rb, int64_t out_rb,
                          double scale, int accumulate) {
  using R = typename Arith<TI, TO>::R;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int rhs = blockIdx.y;
  Spinor<R> x;
  load_spinor_as<TI, R>(in + rhs * in_rb, s, V, x);
  const R sc = R(scale);
#pragma unroll
  for (int k = 0; k < 12; ++k) x.c[k] = sc * x.c[k];
  if (accumulate) {
    Spinor<R> y;
    load_spinor_as<TO, R>(out + rhs * out_rb, s, V, y);
#pragma unroll
    for (int k = 0; k < 12; ++k) x.c[k] = x.c[k] + y.c[k];
  }
  store_spinor_as<TO, R>(out + rhs * out_rb, s, V, x);
}

void launch_convert(OpPrec pi, OpPrec po, const void* in, void* out, int64_t V, int nrhs, double scale,
                    int accumulate, cudaStream_t st) {
  const int64_t irb = (int64_t)spinor_bytes_per_site(pi) * V, orb = (int64_t)spinor_bytes_per_site(po) * V;
  dim3 grid(grid_for(V), nrhs);
  OV_DISPATCH1(pi, TI, {
    OV_DISPATCH1(po, TO, {
      k_convert<TI, TO><<<grid, kThreads, 0, st>>>(static_cast<const char*>(in), static_cast<char*>(out), V, irb,
                                                   orb, scale, accumulate);
    });
  });
}

}  // namespace ov
