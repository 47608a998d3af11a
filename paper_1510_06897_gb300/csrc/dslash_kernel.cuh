// Stencil kernel template (shared by the per-precision translation units
// dslash_f64.cu, dslash_f32.cu, dslash_f16.cu, dslash_b16.cu).
//
//   (D_W x)(s) = 4 x(s) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(s) x(s+mu^)
//                                     + (1 + gamma_mu) U_mu(s-mu^)^dagger x(s-mu^) ]     (Eq. 2)
//   K x        = gamma5 (D_W - m_W) x                                                      (Sec. 2)
//
// One thread per site and right-hand side.  Each of the 8 hops projects the
// neighbour spinor to a two-spinor with (1 -/+ gamma_mu), multiplies the two
// colour vectors by U or U^dagger (reconstructed from 12 reals in FP32/FP16/
// BF16 storage) and expands the result back into the accumulator, so a hop
// costs 2 SU(3) mat-vecs instead of 4.  The paper merges the Wilson matrix with
// the polynomial algebra of the sign function into one kernel (Sec. 2); here
// the merge is the epilogue: out = c0 y + G(s1 r + sum_j w_j v_j), which
// covers plain K, every step of the Chebyshev recurrence and the final
// deflation-correction + overlap assembly (Eq. 1) without extra passes.
//
// Gamma basis: chiral (DeGrand-Rossi), gamma5 = diag(1, 1, -1, -1).  With
// h = (h0, h1) the projected two-spinor, the full spinors are
//   x:  (1-g) psi = (h0, h1,  i h1,  i h0), h = (p0 - i p3, p1 - i p2)
//       (1+g) psi = (h0, h1, -i h1, -i h0), h = (p0 + i p3, p1 + i p2)
//   y:  (1-g) psi = (h0, h1, -h1,  h0),     h = (p0 + p3, p1 - p2)
//       (1+g) psi = (h0, h1,  h1, -h0),     h = (p0 - p3, p1 + p2)
//   z:  (1-g) psi = (h0, h1,  i h0, -i h1), h = (p0 - i p2, p1 + i p3)
//       (1+g) psi = (h0, h1, -i h0,  i h1), h = (p0 + i p2, p1 - i p3)
//   t:  (1-g) psi = (h0, h1, -h0, -h1),     h = (p0 - p2, p1 - p3)
//       (1+g) psi = (h0, h1,  h0,  h1),     h = (p0 + p2, p1 + p3)
#pragma once
#include <utility>
#include "common.cuh"
#include "internal.h"
#include "spin.cuh"

namespace ov {

// 16-bit spinors are projected in packed arithmetic (see spin.cuh).
template <class ST>
constexpr bool kPacked16 = std::is_same<ST, F16>::value || std::is_same<ST, B16>::value;

// Accumulation of one projected, multiplied hop: paired FP32 additions for
// FP32 accumulators, scalar ones for FP64; sg is the sign of a t hop.
template <int MU, int SIGN, class R>
__device__ __forceinline__ void accumulate_hop(Spinor<R>& acc, const Half<R>& uh, R sg) {
  if constexpr (std::is_same<R, float>::value) {
    if constexpr (MU == 3) expand_add_t2<SIGN>(acc, uh, sg);
    else expand_add2<MU, SIGN>(acc, uh);
  } else {
    if constexpr (MU == 3) expand_add_t<SIGN>(acc, uh, sg);
    else expand_add<MU, SIGN>(acc, uh);
  }
}

// Both hops of direction MU for site s and the RT right-hand sides of this
// thread (fields rhs_bytes apart, the last nv of them valid): the link of
// each hop is loaded (and rebuilt) once and applied to every right-hand side.
// n_f / n_b are the neighbour indices; neg_f / neg_b flip the sign (-1
// across an antiperiodic t boundary).  16-bit storage keeps the link and the
// projected two-spinor as packed words whose halves feed the FP32 FMAs
// directly (mul_u16 / mul_udag16).
template <int MU, class LT, int LREC, class ST, int RT, class R>
__device__ __forceinline__ void hop_pair(int s, int n_f, int n_b, bool neg_f, bool neg_b, int V, const void* links,
                                         const char* in, long long rhs_bytes, int nv, Spinor<R> (&acc)[RT]) {
  const R sg_f = neg_f ? R(-1) : R(1), sg_b = neg_b ? R(-1) : R(1);  // used by the t hops only
  if constexpr (kPacked16<ST>) {
    static_assert(std::is_same<LT, ST>::value, "16-bit spinors come with 16-bit links of the same type");
    {  // forward: (1 - gamma_mu) U_mu(s) x(s + mu^)
      uint32_t uw[9];
      load_link_words16<LT, LREC>(links, MU, s, V, uw);
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        if (RT == 1 || r < nv) {
          uint32_t w[12], hw[6];
          load_words16(in + r * rhs_bytes, n_f, V, w);
          project16w<MU, -1, ST>(w, hw);
          Half<float> uh;
          mul_u16<ST>(uw, hw, uh);
          accumulate_hop<MU, -1>(acc[r], uh, sg_f);
        }
      }
    }
    {  // backward: (1 + gamma_mu) U_mu(s - mu^)^dagger x(s - mu^)
      uint32_t uw[9];
      load_link_words16<LT, LREC>(links, MU, n_b, V, uw);
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        if (RT == 1 || r < nv) {
          uint32_t w[12], hw[6];
          load_words16(in + r * rhs_bytes, n_b, V, w);
          project16w<MU, +1, ST>(w, hw);
          Half<float> uh;
          mul_udag16<ST>(uw, hw, uh);
          accumulate_hop<MU, +1>(acc[r], uh, sg_b);
        }
      }
    }
  } else {
    {  // forward: (1 - gamma_mu) U_mu(s) x(s + mu^)
      SU3<R> u;
      load_link<LT, R>(links, MU, s, V, u);
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        if (RT == 1 || r < nv) {  // RT = 1: every launched thread has its right-hand side
          Half<R> h, uh;
          Spinor<R> p;
          load_spinor_as<ST, R>(in + r * rhs_bytes, n_f, V, p);
          project<MU, -1>(p, h);
          mul_u(u, h, uh);
          accumulate_hop<MU, -1>(acc[r], uh, sg_f);
        }
      }
    }
    {  // backward: (1 + gamma_mu) U_mu(s - mu^)^dagger x(s - mu^)
      SU3<R> u;
      load_link<LT, R>(links, MU, n_b, V, u);
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        if (RT == 1 || r < nv) {
          Half<R> h, uh;
          Spinor<R> p;
          load_spinor_as<ST, R>(in + r * rhs_bytes, n_b, V, p);
          project<MU, +1>(p, h);
          mul_udag(u, h, uh);
          accumulate_hop<MU, +1>(acc[r], uh, sg_b);
        }
      }
    }
  }
}

// Epilogue coefficients in the arithmetic type R, formed once on the host
// (a per-thread FP64 conversion would occupy the slow FP64 pipe) with every
// sign folded in: index [0] applies to spins 0, 1 and [1] to spins 2, 3.
//   out = xa x + ha acc + sum_j w_j v_j + wz z + c0 y
// equals c0 y + G5(s1 G (d x - acc / 2) + sum_j w_j v_j + wz z) with G =
// gamma5 for K (1 for D_W), d = 4 - m_w (4 for D_W), G5 = gamma5 if g5_out,
// and acc the hop sum.
template <class R>
struct EpiDev {
  R xa[2], ha[2];
  R w[3][2];
  R wz[2];
  R c0;
  const void* v[3];
  const void* z;
  const void* y;
};

// Epilogue of one site and right-hand side (fields at byte offsets off / ooff).
template <class ST, class OT, class R>
__device__ __forceinline__ void epilogue(const EpiDev<R>& e, const char* in, char* out, int s, int V, long long off,
                                         long long ooff, const Spinor<R>& acc) {
  Spinor<R> xs;
  load_spinor_as<ST, R>(in + off, s, V, xs);
  Spinor<R> r;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int h = k < 6 ? 0 : 1;
    r.c[k] = {fma_(e.xa[h], xs.c[k].re, e.ha[h] * acc.c[k].re), fma_(e.xa[h], xs.c[k].im, e.ha[h] * acc.c[k].im)};
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (e.v[j] != nullptr) {
      Spinor<R> vj;
      load_spinor_as<ST, R>(static_cast<const char*>(e.v[j]) + off, s, V, vj);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const R wj = e.w[j][k < 6 ? 0 : 1];
        r.c[k] = {fma_(wj, vj.c[k].re, r.c[k].re), fma_(wj, vj.c[k].im, r.c[k].im)};
      }
    }
  }
  if (e.z != nullptr) {
    Spinor<R> zv;
    load_spinor_as<OT, R>(static_cast<const char*>(e.z) + ooff, s, V, zv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R wz = e.wz[k < 6 ? 0 : 1];
      r.c[k] = {fma_(wz, zv.c[k].re, r.c[k].re), fma_(wz, zv.c[k].im, r.c[k].im)};
    }
  }
  if (e.y != nullptr) {
    Spinor<R> yv;
    load_spinor_as<OT, R>(static_cast<const char*>(e.y) + ooff, s, V, yv);
#pragma unroll
    for (int k = 0; k < 12; ++k) r.c[k] = {fma_(e.c0, yv.c[k].re, r.c[k].re), fma_(e.c0, yv.c[k].im, r.c[k].im)};
  }
  store_spinor_as<OT, R>(out + ooff, s, V, r);
}

struct Geo {
  int L[4];
  int V;
  int LxLy;
  int antiperiodic_t;
  int brick_z;  // 0: a block covers consecutive sites of one (x, y) plane; > 0: an 8 x 4 x brick_z brick
};

// Site coordinates of this thread.  Plane mapping: grid x runs over the
// sites of an (x, y) plane, grid y over the (z, t) slices.  Brick mapping:
// a block of 32 brick_z threads covers an 8 x 4 x brick_z brick of one t
// slice (grid x: bricks of the (x, y, z) volume, grid y: t), so that more of
// the z and y neighbours a block reads are its own sites, whose lines the
// block's other loads already brought into L1.  Returns false for the
// padding threads of a plane.
__device__ __forceinline__ bool site_of_thread(const Geo& g, int& x, int& y, int& z, int& t) {
  const int Lx = g.L[0], Lz = g.L[2];
  if (g.brick_z > 0) {
    const int tid = threadIdx.x;
    const int nbx = Lx >> 3, nby = g.L[1] >> 2;
    const int b = blockIdx.x;
    const int bxi = b % nbx, r = b / nbx;
    const int byi = r % nby, bzi = r / nby;
    x = (bxi << 3) + (tid & 7);
    y = (byi << 2) + ((tid >> 3) & 3);
    z = bzi * g.brick_z + (tid >> 5);
    t = blockIdx.y;
    return true;
  }
  const int xy = blockIdx.x * blockDim.x + threadIdx.x;
  if (xy >= g.LxLy) return false;
  const int slice = blockIdx.y;
  y = xy / Lx;
  x = xy - y * Lx;
  t = slice / Lz;
  z = slice - t * Lz;
  return true;
}

// Grid of a stencil launch for either mapping (z: right-hand-side tiles).
inline dim3 stencil_grid(const Geo& g, int tpb, unsigned ztiles) {
  if (g.brick_z > 0)
    return dim3((unsigned)((g.L[0] / 8) * (g.L[1] / 4) * (g.L[2] / g.brick_z)), (unsigned)g.L[3], ztiles);
  return dim3((unsigned)((g.LxLy + tpb - 1) / tpb), (unsigned)(g.L[2] * g.L[3]), ztiles);
}



// Grid: x = sites of one (x, y) plane, y = z + Lz t slice, z = tile of RT
// right-hand sides.  LT/LREC: link storage and 12- or 18-real layout, ST:
// storage of the stencil input and of v[j], OT: storage of z, y and the
// output.  MINB: minimum resident blocks of 256 threads requested from the
// register allocator (1: no cap, 2: <= 128 registers, 3: <= 80, 4: <= 64),
// or (MINB 5) 14 resident blocks of at most 64 threads (<= 72 registers):
// an occupancy between the 256-thread caps that lets the number of waves of
// a launch end closer to a whole number (4.87 instead of 4.26 on 24^3 x 48).
constexpr int lb_threads(int minb) { return minb == 5 ? 64 : 256; }
constexpr int lb_blocks(int minb) { return minb == 5 ? 14 : minb; }
// Programmatic dependent launch: a stencil launched with the
// programmatic-stream-serialisation attribute may start while the previous
// kernel of the stream drains; it lets its own dependents start likewise and
// waits for the previous kernel to complete (and its writes to be visible)
// before its first global access.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

template <class LT, int LREC, class ST, class OT, int MINB, int RT>
__global__ void __launch_bounds__(lb_threads(MINB), lb_blocks(MINB)) k_dslash(Geo g, const void* __restrict__ links,
                                                      const char* __restrict__ in, char* out, EpiDev<typename Store<ST>::R> e,
                                                      long long rhs_bytes, long long out_rhs_bytes, int nrhs) {
  using R = typename Store<ST>::R;
  pdl_enter();
  int x, y, z, t;
  if (!site_of_thread(g, x, y, z, t)) return;
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  const int s = (t * Lz + z) * g.LxLy + y * Lx + x;
  const int V = g.V;
  const int r0 = blockIdx.z * RT;
  const int nv = min(RT, nrhs - r0);
  const char* xin = in + (long long)r0 * rhs_bytes;

  const int sz = g.LxLy, st = g.LxLy * Lz;
  const int xp = (x == Lx - 1) ? s - (Lx - 1) : s + 1;
  const int xm = (x == 0) ? s + (Lx - 1) : s - 1;
  const int yp = (y == Ly - 1) ? s - (Ly - 1) * Lx : s + Lx;
  const int ym = (y == 0) ? s + (Ly - 1) * Lx : s - Lx;
  const int zp = (z == Lz - 1) ? s - (Lz - 1) * sz : s + sz;
  const int zm = (z == 0) ? s + (Lz - 1) * sz : s - sz;
  const int tp = (t == Lt - 1) ? s - (Lt - 1) * st : s + st;
  const int tm = (t == 0) ? s + (Lt - 1) * st : s - st;
  const bool neg_tf = g.antiperiodic_t && t == Lt - 1;  // antiperiodic wrap of the t hops
  const bool neg_tb = g.antiperiodic_t && t == 0;

  Spinor<R> acc[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[r].c[k] = {R(0), R(0)};
  hop_pair<0, LT, LREC, ST, RT, R>(s, xp, xm, false, false, V, links, xin, rhs_bytes, nv, acc);
  hop_pair<1, LT, LREC, ST, RT, R>(s, yp, ym, false, false, V, links, xin, rhs_bytes, nv, acc);
  hop_pair<2, LT, LREC, ST, RT, R>(s, zp, zm, false, false, V, links, xin, rhs_bytes, nv, acc);
  hop_pair<3, LT, LREC, ST, RT, R>(s, tp, tm, neg_tf, neg_tb, V, links, xin, rhs_bytes, nv, acc);

#pragma unroll
  for (int rr = 0; rr < RT; ++rr) {
    if (RT > 1 && rr >= nv) break;
    epilogue<ST, OT>(e, in, out, s, V, (long long)(r0 + rr) * rhs_bytes, (long long)(r0 + rr) * out_rhs_bytes,
                     acc[rr]);
  }
}

inline Geo make_geo(const LatticeH& gh) {
  Geo g;
  for (int i = 0; i < 4; ++i) g.L[i] = gh.L[i];
  g.V = (int)gh.V;
  g.LxLy = gh.L[0] * gh.L[1];
  g.antiperiodic_t = gh.antiperiodic_t;
  g.brick_z = 0;
  return g;
}

template <class R>
inline EpiDev<R> make_epi(const EpiArgs& ea) {
  const double g_lo = ea.wilson ? 1.0 : -1.0;  // G on spins 2, 3
  const double o_lo = ea.g5_out ? -1.0 : 1.0;  // G5 on spins 2, 3
  const double d = ea.wilson ? 4.0 : 4.0 - ea.m_w;
  EpiDev<R> e;
  e.xa[0] = R(ea.s1 * d);
  e.xa[1] = R(ea.s1 * d * g_lo * o_lo);
  e.ha[0] = R(-0.5 * ea.s1);
  e.ha[1] = R(-0.5 * ea.s1 * g_lo * o_lo);
  for (int j = 0; j < 3; ++j) {
    e.v[j] = ea.v[j];
    e.w[j][0] = R(ea.w[j]);
    e.w[j][1] = R(ea.w[j] * o_lo);
  }
  e.z = ea.z;
  e.wz[0] = R(ea.wz);
  e.wz[1] = R(ea.wz * o_lo);
  e.y = ea.y;
  e.c0 = R(ea.c0);
  if (ea.keep_half == 0 || ea.keep_half == 1) {  // chiral projection of everything but c0 y
    const int h = 1 - ea.keep_half;
    e.xa[h] = e.ha[h] = e.wz[h] = R(0);
    for (int j = 0; j < 3; ++j) e.w[j][h] = R(0);
  }
  return e;
}

// Whether stencil launches overlap the previous kernel's drain (programmatic
// dependent launch; OV_PDL=0 turns it off).
bool pdl_enabled();

// Launches kern<<<grid, block, smem, st>>>(args...), with the persisting L2
// window on the links when one is set for this links pointer, and with
// programmatic dependent launch when pdl is set (kernels that call
// pdl_enter() before any global access).
template <class... KA, class... A>
void launch_windowed(void (*kern)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, const void* links,
                     bool pdl, A&&... args) {
  const L2Window& w = l2_window();
  const bool window = (w.base != nullptr && w.base == links);
  if (window || pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int n = 0;
    if (window) {
      attr[n].id = cudaLaunchAttributeAccessPolicyWindow;
      attr[n].val.accessPolicyWindow.base_ptr = const_cast<void*>(w.base);
      attr[n].val.accessPolicyWindow.num_bytes = w.bytes;
      attr[n].val.accessPolicyWindow.hitRatio = 1.0f;
      attr[n].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
      attr[n].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
      ++n;
    }
    if (pdl) {
      attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[n].val.programmaticStreamSerializationAllowed = 1;
      ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
    return;
  }
  kern<<<grid, block, smem, st>>>(std::forward<A>(args)...);
}

template <class LT, int LREC, class ST, class OT, int MINB, int RT>
void launch_k(const LatticeH& gh, const void* links, const void* in, void* out, const EpiArgs& ea, int nrhs, int tpb,
              bool brick, cudaStream_t st) {
  Geo g = make_geo(gh);
  if (brick) g.brick_z = tpb / 32;
  const long long rb = (long long)Store<ST>::bytes_per_site * g.V, orb = (long long)Store<OT>::bytes_per_site * g.V;
  const dim3 grid = stencil_grid(g, tpb, (unsigned)((nrhs + RT - 1) / RT));
  launch_windowed(k_dslash<LT, LREC, ST, OT, MINB, RT>, grid, dim3(tpb), 0, st, links, pdl_enabled(), g, links,
                  static_cast<const char*>(in), static_cast<char*>(out), make_epi<typename Store<ST>::R>(ea), rb, orb,
                  nrhs);
}

// Variant table: (minb, rt) pairs compiled for each storage combination.
template <class LT, int LREC, class ST, class OT>
bool launch_variant(const DslashCfg& c, const LatticeH& g, const void* links, const void* in, void* out,
                    const EpiArgs& e, int nrhs, cudaStream_t st) {
  if (c.brick && !brick_lattice_ok(g, c.tpb)) return false;
#define OV_V(MB, RTV)                                                                 \
  if (c.minb == MB && c.rt == RTV) {                                                  \
    launch_k<LT, LREC, ST, OT, MB, RTV>(g, links, in, out, e, nrhs, c.tpb, c.brick != 0, st); \
    return true;                                                                      \
  }
  if (c.minb >= 5 && c.tpb > 64) return false;  // these caps are compiled for blocks of <= 64 threads
  OV_V(2, 1) OV_V(3, 1) OV_V(4, 1) OV_V(5, 1)
  if constexpr (!std::is_same<ST, F64>::value) {
    OV_V(2, 2) OV_V(3, 2) OV_V(1, 3) OV_V(2, 3) OV_V(1, 4) OV_V(2, 4) OV_V(1, 6)
  }
#undef OV_V
  return false;
}

}  // namespace ov
