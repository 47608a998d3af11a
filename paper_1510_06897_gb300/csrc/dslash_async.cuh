// Staged variant of the stencil of Eq. 2 for 16-bit storage with
// reconstruct-12 links (one right-hand side per thread).
//
// The gather kernel (dslash_kernel.cuh) loads each hop's neighbour spinor and
// link into registers right before using them, so a thread waits on memory
// once per direction, and at 64 registers a scheduler holds too few warps to
// cover those waits (the FMA pipe sits idle ~40% of a launch).  Here every
// thread copies the operands of the next direction into its own slots of
// shared memory with asynchronous copies (cp.async, 16 B per spinor chunk,
// 8 B per link chunk) while it computes the current one, double-buffered
// over the four directions:
//
//   issue x -> buf 0, y -> buf 1
//   wait x, hops x, issue z -> buf 0
//   wait y, hops y, issue t -> buf 1
//   wait z, hops z, issue the epilogue vectors x(s), v_0, v_1 -> buf 0
//   wait t, hops t, issue v_2 -> buf 1
//   wait, epilogue
//
// A copy in flight holds no register.  A thread reads only the slots it
// filled itself, so no barrier is needed: cp.async.wait_group makes a
// thread's own completed copies visible to it, and a slot is refilled only
// after the instructions that consumed its previous contents have issued.
// The arithmetic is that of the gather kernel in the same order, so the two
// variants give bit-identical results.
//
// Shared memory per thread: 2 buffers x (6 spinor chunks of 16 B + 6 link
// chunks of 8 B) = 288 B (STAGE_LINKS = 1), or 192 B with the links loaded
// from global memory as in the gather kernel (STAGE_LINKS = 0).
#pragma once
#include "dslash_kernel.cuh"

namespace ov {

namespace asy {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Zero that the compiler cannot see through, computed from two hop sums:
// added to the shared address of a refill, it makes the refill wait until
// those sums exist, i.e. until every word read from the buffer being
// refilled has arrived in registers.  (acc components 2 and 5 -- spins 0 and
// 1, colour 2 -- depend on all twelve spinor words of both hops through the
// two spin projections and on all link words through the rebuilt row 2.)
__device__ __forceinline__ uint32_t after(const Spinor<float>& acc) {
  uint32_t z;
  asm volatile("{\n .reg .b32 t;\n xor.b32 t, %1, %2;\n and.b32 %0, t, 0;\n}"
               : "=r"(z)
               : "r"(__float_as_uint(acc.c[2].re)), "r"(__float_as_uint(acc.c[5].re)));
  return z;
}
template <int N>
__device__ __forceinline__ void wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The block's shared memory (dynamic): spinor chunk k (0..5) of buffer b for
// thread tid at uint4 index (b * 6 + k) * T + tid; after the 192 T bytes of
// spinor slots, link chunk k of buffer b at uint2 index (b * 6 + k) * T + tid.
// A buffer's link area (6 x 8 B) also holds one 16-bit spinor (3 x 16 B) at
// uint4 index (b * 3 + k) * T + tid of that area.
extern __shared__ __align__(16) unsigned char async_smem[];

struct Slots {
  int T, tid;
  uint32_t base;  // shared-window address of async_smem
  __device__ uint32_t spin_addr(int b, int k) const { return base + (uint32_t)(((b * 6 + k) * T + tid) * 16); }
  __device__ uint32_t link_addr(int b, int k) const {
    return base + (uint32_t)(192 * T) + (uint32_t)(((b * 6 + k) * T + tid) * 8);
  }
  __device__ uint32_t link16_addr(int b, int k) const {
    return base + (uint32_t)(192 * T) + (uint32_t)(((b * 3 + k) * T + tid) * 16);
  }
  __device__ void words(int b, int k0, uint32_t (&w)[12]) const {  // 3 spinor chunks from k0
    const uint4* sp = reinterpret_cast<const uint4*>(async_smem);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 v = sp[(b * 6 + k0 + c) * T + tid];
      w[4 * c] = v.x;
      w[4 * c + 1] = v.y;
      w[4 * c + 2] = v.z;
      w[4 * c + 3] = v.w;
    }
  }
  __device__ void words16(int b, uint32_t (&w)[12]) const {  // the spinor held in a link area
    const uint4* sp = reinterpret_cast<const uint4*>(async_smem + 192 * T);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 v = sp[(b * 3 + c) * T + tid];
      w[4 * c] = v.x;
      w[4 * c + 1] = v.y;
      w[4 * c + 2] = v.z;
      w[4 * c + 3] = v.w;
    }
  }
  __device__ void link_words(int b, int k0, uint32_t (&uw)[9]) const {  // rows 0, 1 of a 12-real link
    const uint2* lp = reinterpret_cast<const uint2*>(async_smem + 192 * T);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint2 v = lp[(b * 6 + k0 + c) * T + tid];
      uw[2 * c] = v.x;
      uw[2 * c + 1] = v.y;
    }
  }
};

// The 3 chunks of a 16-bit spinor (site n of field p) into 3 consecutive slots.
__device__ __forceinline__ void issue_spinor(uint32_t dst0, uint32_t stride, const void* p, int n, int V) {
  const uint4* q = static_cast<const uint4*>(p);
#pragma unroll
  for (int c = 0; c < 3; ++c) cp16(dst0 + c * stride, q + (int64_t)c * V + n);
}

// The operands of direction mu into buffer b (dep: see after()).
template <int SL>
__device__ __forceinline__ void issue_direction(const Slots& sl, int b, int mu, int s, int nf, int nb, const void* in,
                                                const void* links, int V, uint32_t dep) {
  const uint32_t st16 = (uint32_t)sl.T * 16u;
  issue_spinor(sl.spin_addr(b, 0) + dep, st16, in, nf, V);
  issue_spinor(sl.spin_addr(b, 3) + dep, st16, in, nb, V);
  if constexpr (SL) {
    const uint2* q = static_cast<const uint2*>(links) + (int64_t)mu * 3 * V;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cp8(sl.link_addr(b, c) + dep, q + (int64_t)c * V + s);
      cp8(sl.link_addr(b, 3 + c) + dep, q + (int64_t)c * V + nb);
    }
  }
  commit();
}

// Both hops of direction MU from buffer b: the same operations, in the same
// order, as hop_pair of the gather kernel with one right-hand side.
template <int MU, class ST, int SL>
__device__ __forceinline__ void hops_from_slots(const Slots& sl, int b, int s, int nb, int V, const void* links,
                                                float sg_f, float sg_b, Spinor<float>& acc) {
  {  // forward: (1 - gamma_mu) U_mu(s) x(s + mu^)
    uint32_t uw[9];
    if constexpr (SL) {
      sl.link_words(b, 0, uw);
      reconstruct16<ST>(uw);
    } else {
      load_link_words16<ST, 12>(links, MU, s, V, uw);
    }
    uint32_t w[12], hw[6];
    sl.words(b, 0, w);
    project16w<MU, -1, ST>(w, hw);
    Half<float> uh;
    mul_u16<ST>(uw, hw, uh);
    accumulate_hop<MU, -1>(acc, uh, sg_f);
  }
  {  // backward: (1 + gamma_mu) U_mu(s - mu^)^dagger x(s - mu^)
    uint32_t uw[9];
    if constexpr (SL) {
      sl.link_words(b, 3, uw);
      reconstruct16<ST>(uw);
    } else {
      load_link_words16<ST, 12>(links, MU, nb, V, uw);
    }
    uint32_t w[12], hw[6];
    sl.words(b, 3, w);
    project16w<MU, +1, ST>(w, hw);
    Half<float> uh;
    mul_udag16<ST>(uw, hw, uh);
    accumulate_hop<MU, +1>(acc, uh, sg_b);
  }
}

template <class ST>
__device__ __forceinline__ void words_to_spinor(const uint32_t (&w)[12], Spinor<float>& o) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 f = unpack2<ST>(w[k]);
    o.c[k] = {f.x, f.y};
  }
}

// Where the epilogue's 16-bit vectors (x(s), then the non-null v_j in order)
// are staged: index i < na goes to group A (buffer 0, issued after the z
// hops), the rest to group B (buffer 1, issued after the t hops).  Slot
// numbers within a buffer: 0 = spinor chunks 0..2, 1 = chunks 3..5, 2 = the
// link area (only with staged links).
template <int SL>
struct EpiPlan {
  static constexpr int na = SL ? 3 : 2;
  __device__ static int buf(int i) { return i < na ? 0 : 1; }
  __device__ static int slot(int i) { return i < na ? i : i - na; }
};

template <int SL>
__device__ __forceinline__ void issue_epi_vec(const Slots& sl, int i, const void* p, int n, int V, uint32_t dep) {
  const int b = EpiPlan<SL>::buf(i), k = EpiPlan<SL>::slot(i);
  if (k == 2)
    issue_spinor(sl.link16_addr(b, 0) + dep, (uint32_t)sl.T * 16u, p, n, V);
  else
    issue_spinor(sl.spin_addr(b, 3 * k) + dep, (uint32_t)sl.T * 16u, p, n, V);
}

// Stages the epilogue's 16-bit vectors with index in [lo, hi): index 0 is
// x(s), then the non-null v_j in order (off: the right-hand side's offset).
template <int SL>
__device__ __forceinline__ void issue_epi_range(const Slots& sl, int lo, int hi, const char* xin,
                                                const EpiDev<float>& e, long long off, int s, int V, uint32_t dep) {
  int i = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const void* p = (j == 0) ? static_cast<const void*>(xin)
                             : (e.v[j - 1] != nullptr ? static_cast<const void*>(
                                                            static_cast<const char*>(e.v[j - 1]) + off)
                                                      : nullptr);
    if (p != nullptr) {
      if (i >= lo && i < hi) issue_epi_vec<SL>(sl, i, p, s, V, dep);
      ++i;
    }
  }
  commit();
}

template <int SL>
__device__ __forceinline__ void read_epi_vec(const Slots& sl, int i, uint32_t (&w)[12]) {
  const int b = EpiPlan<SL>::buf(i), k = EpiPlan<SL>::slot(i);
  if (k == 2)
    sl.words16(b, w);
  else
    sl.words(b, 3 * k, w);
}

}  // namespace asy

// Grid and block as the gather kernel with one right-hand side per thread
// (x: sites of an (x, y) plane, y: (z, t) slice, z: right-hand side).
template <class ST, class OT, int MINB, int SL>
__global__ void __launch_bounds__(256, MINB)
    k_dslash_async(Geo g, const void* __restrict__ links, const char* __restrict__ in, char* out, EpiDev<float> e,
                   long long rhs_bytes, long long out_rhs_bytes) {
  pdl_enter();
  const int T = blockDim.x, tid = threadIdx.x;
  int x, y, z, t;
  if (!site_of_thread(g, x, y, z, t)) return;  // no barrier below: every thread works on its own slots only
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  const int s = (t * Lz + z) * g.LxLy + y * Lx + x;
  const int V = g.V;
  const long long off = (long long)blockIdx.z * rhs_bytes, ooff = (long long)blockIdx.z * out_rhs_bytes;
  const char* xin = in + off;

  const int sz = g.LxLy, stt = g.LxLy * Lz;
  const int xp = (x == Lx - 1) ? s - (Lx - 1) : s + 1;
  const int xm = (x == 0) ? s + (Lx - 1) : s - 1;
  const int yp = (y == Ly - 1) ? s - (Ly - 1) * Lx : s + Lx;
  const int ym = (y == 0) ? s + (Ly - 1) * Lx : s - Lx;
  const int zp = (z == Lz - 1) ? s - (Lz - 1) * sz : s + sz;
  const int zm = (z == 0) ? s + (Lz - 1) * sz : s - sz;
  const int tp = (t == Lt - 1) ? s - (Lt - 1) * stt : s + stt;
  const int tm = (t == 0) ? s + (Lt - 1) * stt : s - stt;
  const float sg_tf = (g.antiperiodic_t && t == Lt - 1) ? -1.f : 1.f;
  const float sg_tb = (g.antiperiodic_t && t == 0) ? -1.f : 1.f;

  asy::Slots sl;
  sl.T = T;
  sl.tid = tid;
  sl.base = asy::smem_u32(asy::async_smem);

  constexpr int na = asy::EpiPlan<SL>::na;
  asy::issue_direction<SL>(sl, 0, 0, s, xp, xm, xin, links, V, 0u);
  asy::issue_direction<SL>(sl, 1, 1, s, yp, ym, xin, links, V, 0u);

  Spinor<float> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = {0.f, 0.f};

  asy::wait_group<1>();
  asy::hops_from_slots<0, ST, SL>(sl, 0, s, xm, V, links, 1.f, 1.f, acc);
  asy::issue_direction<SL>(sl, 0, 2, s, zp, zm, xin, links, V, asy::after(acc));
  asy::wait_group<1>();
  asy::hops_from_slots<1, ST, SL>(sl, 1, s, ym, V, links, 1.f, 1.f, acc);
  asy::issue_direction<SL>(sl, 1, 3, s, tp, tm, xin, links, V, asy::after(acc));
  asy::wait_group<1>();
  asy::hops_from_slots<2, ST, SL>(sl, 0, s, zm, V, links, 1.f, 1.f, acc);
  asy::issue_epi_range<SL>(sl, 0, na, xin, e, off, s, V, asy::after(acc));
  asy::wait_group<1>();
  asy::hops_from_slots<3, ST, SL>(sl, 1, s, tm, V, links, sg_tf, sg_tb, acc);
  asy::issue_epi_range<SL>(sl, na, 4, xin, e, off, s, V, asy::after(acc));

  // epilogue: the operations of epilogue() in the same order
  asy::wait_group<1>();
  Spinor<float> r;
  {
    uint32_t w[12];
    asy::read_epi_vec<SL>(sl, 0, w);
    Spinor<float> xs;
    asy::words_to_spinor<ST>(w, xs);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int h = k < 6 ? 0 : 1;
      r.c[k] = {fma_(e.xa[h], xs.c[k].re, e.ha[h] * acc.c[k].re), fma_(e.xa[h], xs.c[k].im, e.ha[h] * acc.c[k].im)};
    }
  }
  int i = 1;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (e.v[j] != nullptr) {
      if (i == na) asy::wait_group<0>();
      uint32_t w[12];
      asy::read_epi_vec<SL>(sl, i, w);
      Spinor<float> vj;
      asy::words_to_spinor<ST>(w, vj);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float wj = e.w[j][k < 6 ? 0 : 1];
        r.c[k] = {fma_(wj, vj.c[k].re, r.c[k].re), fma_(wj, vj.c[k].im, r.c[k].im)};
      }
      ++i;
    }
  }
  if (e.z != nullptr) {
    Spinor<float> zv;
    load_spinor_as<OT, float>(static_cast<const char*>(e.z) + ooff, s, V, zv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float wz = e.wz[k < 6 ? 0 : 1];
      r.c[k] = {fma_(wz, zv.c[k].re, r.c[k].re), fma_(wz, zv.c[k].im, r.c[k].im)};
    }
  }
  if (e.y != nullptr) {
    Spinor<float> yv;
    load_spinor_as<OT, float>(static_cast<const char*>(e.y) + ooff, s, V, yv);
#pragma unroll
    for (int k = 0; k < 12; ++k) r.c[k] = {fma_(e.c0, yv.c[k].re, r.c[k].re), fma_(e.c0, yv.c[k].im, r.c[k].im)};
  }
  store_spinor_as<OT, float>(out + ooff, s, V, r);
}

// Dynamic shared memory of one block of tpb threads.
inline size_t async_smem_bytes(int tpb, int stage_links) { return (size_t)tpb * (stage_links ? 288 : 192); }

template <class ST, class OT, int MINB, int SL>
bool launch_async_k(const LatticeH& gh, const void* links, const void* in, void* out, const EpiArgs& ea, int nrhs,
                    int tpb, bool brick, cudaStream_t st) {
  auto kern = k_dslash_async<ST, OT, MINB, SL>;
  const size_t smem = async_smem_bytes(tpb, SL);
  static bool attr_set = false;  // per instantiation; the largest block size is set once
  if (!attr_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)async_smem_bytes(256, SL)) !=
        cudaSuccess)
      return false;
    attr_set = true;
  }
  Geo g = make_geo(gh);
  if (brick) g.brick_z = tpb / 32;
  const long long rb = (long long)Store<ST>::bytes_per_site * g.V, orb = (long long)Store<OT>::bytes_per_site * g.V;
  const dim3 grid = stencil_grid(g, tpb, (unsigned)nrhs);
  launch_windowed(kern, grid, dim3(tpb), smem, st, links, pdl_enabled(), g, links, static_cast<const char*>(in),
                  static_cast<char*>(out), make_epi<float>(ea), rb, orb);
  return true;
}

// The staged variant for storage ST (16-bit, 12-real links): c.async = 1
// stages spinors and links, 2 spinors only; register cap as c.minb (3 or 4).
template <class ST, class OT>
bool launch_async(const DslashCfg& c, const LatticeH& g, const void* links, const void* in, void* out,
                  const EpiArgs& e, int nrhs, cudaStream_t st) {
  if (c.lrec != 12 || c.rt != 1 || c.tpb > 256) return false;
  if (c.brick && !brick_lattice_ok(g, c.tpb)) return false;
  const bool bk = c.brick != 0;
  const int sl = c.async == 1 ? 1 : 0;
  if (c.minb == 3) {
    return sl ? launch_async_k<ST, OT, 3, 1>(g, links, in, out, e, nrhs, c.tpb, bk, st)
              : launch_async_k<ST, OT, 3, 0>(g, links, in, out, e, nrhs, c.tpb, bk, st);
  }
  if (c.minb == 4) {
    return sl ? launch_async_k<ST, OT, 4, 1>(g, links, in, out, e, nrhs, c.tpb, bk, st)
              : launch_async_k<ST, OT, 4, 0>(g, links, in, out, e, nrhs, c.tpb, bk, st);
  }
  return false;
}

}  // namespace ov
