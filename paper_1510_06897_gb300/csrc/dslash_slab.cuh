// Slab variant of the stencil of Eq. 2 for 16-bit storage with
// reconstruct-12 links.  A persistent CTA takes one (z, t) plane of Lx Ly
// sites at a time (one compute thread per site) and applies the eight hops in
// five phases that read only shared memory:
//   XY: the plane's spinors and its U_x, U_y links (four hops);
//   Z+: the spinors of plane z+1 and U_z(z);    Z-: plane z-1 and U_z(z-1);
//   T+: the spinors of plane t+1 and U_t(t);    T-: plane t-1 and U_t(t-1),
//       then the epilogue of the gather kernel.
// In the SoA layout each of these operands is a contiguous run of Lx Ly
// entries per storage chunk, so a phase's operands are a few 1-D bulk copies
// (cp.async.bulk) into one slot of a ring in shared memory.  One producer
// warp issues the copies (a "full" mbarrier per slot counts their bytes) and
// refills a slot once every compute warp has released it (an "empty"
// mbarrier per slot); the compute warps never synchronise with each other,
// so a warp that waits on an epilogue load does not hold the others back.
// The hop sum stays in registers across the five phases of a plane.
// Neighbouring planes are read from L2 by the CTAs working on the adjacent
// slices at about the same time.  Every mbarrier wait is bounded; on expiry
// the warp records an error flag and stops, and the producer waits (bounded)
// for its copies in flight before it exits.
#pragma once
#include "dslash_kernel.cuh"

namespace ov {

namespace slab {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// try_wait may suspend the thread until the phase completes or this many
// nanoseconds pass, so a waiting warp takes no issue slots.
constexpr uint32_t kSuspendHintNs = 10000000;

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity to complete; false after about a
// second (2^31 clocks).  stall (testing, see ov_test_wait_expiry): a device
// flag that nothing sets; when given, the wait first waits up to stall_cycles
// for it, runs out and reports failure as an expired wait would.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* stall = nullptr,
                                          long long stall_cycles = 0) {
  const long long t0 = clock64();
  if (stall != nullptr) {
    while (*stall == 0) {
      if (clock64() - t0 > stall_cycles) return false;
    }
  }
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

// 1-D bulk copy global -> this CTA's shared memory; bytes and both addresses
// multiples of 16.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Threads per CTA at most: the compute threads (one per site of a plane) and
// the producer warp; register budget 65536 / 640 -> 96 per thread.
constexpr int kSlabMaxThreads = 640;
constexpr int kSlabMaxSlots = 4;

// One slot (P = Lx Ly sites): a spinor plane of 3 chunks x P x 16 B, then two
// link planes of 3 chunks x P x 8 B (the second used by phase XY only).
inline size_t slab_slot_bytes(int P) { return (size_t)P * (48 + 2 * 24); }
constexpr size_t kSlabSmemLimit = 227 * 1024;
inline int slab_slots(int P) {
  const size_t avail = kSlabSmemLimit - 2 * kSlabMaxSlots * sizeof(unsigned long long);
  return (int)std::min<size_t>(kSlabMaxSlots, avail / slab_slot_bytes(P));
}
inline size_t slab_smem_bytes(int P) {
  return (size_t)slab_slots(P) * slab_slot_bytes(P) + 2 * kSlabMaxSlots * sizeof(unsigned long long);
}

template <class T>
__device__ __forceinline__ void slab_load_link(const unsigned char* plane, int P, int site, SU3<float>& u) {
  const uint2* q = reinterpret_cast<const uint2*>(plane);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const uint2 v = q[c * P + site];
    const float2 a = unpack2<T>(v.x), b = unpack2<T>(v.y);
    u.u[2 * c] = {a.x, a.y};
    u.u[2 * c + 1] = {b.x, b.y};
  }
  reconstruct_row2(u);
}

__device__ __forceinline__ void slab_load_words(const unsigned char* plane, int P, int site, uint32_t (&w)[12]) {
  const uint4* q = reinterpret_cast<const uint4*>(plane);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const uint4 v = q[c * P + site];
    w[4 * c] = v.x;
    w[4 * c + 1] = v.y;
    w[4 * c + 2] = v.z;
    w[4 * c + 3] = v.w;
  }
}

// One hop from shared memory: (1 -/+ gamma_mu) [U or U^dagger] x(neighbour),
// SIGN -1 forward (U at lsite), +1 backward (U^dagger at lsite).
template <int MU, int SIGN, class T>
__device__ __forceinline__ void slab_hop(const unsigned char* sp, const unsigned char* lk, int P, int nsite,
                                         int lsite, bool neg, Spinor<float>& acc) {
  uint32_t w[12];
  slab_load_words(sp, P, nsite, w);
  Half<float> h, uh;
  project16<MU, SIGN, T>(w, h);
  if (neg) scale_half(h, -1.f);
  SU3<float> u;
  slab_load_link<T>(lk, P, lsite, u);
  if constexpr (SIGN < 0) mul_u(u, h, uh);
  else mul_udag(u, h, uh);
  expand_add<MU, SIGN>(acc, uh);
}

// acc += cu * x (spins 0, 1) and cl * x (spins 2, 3), x a 16-bit spinor in shared memory
template <class T>
__device__ __forceinline__ void slab_axpy(const unsigned char* plane, int P, int site, float cu, float cl,
                                          Spinor<float>& acc) {
  uint32_t w[12];
  slab_load_words(plane, P, site, w);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 f = unpack2<T>(w[k]);
    const float c = (k < 6) ? cu : cl;
    acc.c[k].re = fmaf(c, f.x, acc.c[k].re);
    acc.c[k].im = fmaf(c, f.y, acc.c[k].im);
  }
}

// The epilogue of the gather kernel, rewritten so that everything in the
// input's storage enters one accumulator from shared memory:
//   s1 G (d x - H/2) + sum_j w_j v_j = fs G acc,   fs = -s1/2,
//   acc = H + xs2 x + sum_j G (vcu_j | vcl_j) v_j,  xs2 = -2 d,  vc_j = -2 w_j / s1
// (G = gamma5 for K, 1 for D_W; d = 4 - m_w or 4; H the hop sum).  Then
// out = c0 y + G5(fs G acc + wz z), with z, y (output storage) read from
// global memory.  Needs s1 != 0.
struct SlabEpi {
  const void* v[3];  // the non-null v_j, compacted
  float vcu[3], vcl[3];
  int nv;
  float xs2, fs;
  int kgamma;  // 1: K (G = gamma5), 0: D_W
  const void* z;
  float wz;
  int g5_out;
  const void* y;
  float c0;
};

inline bool slab_epi(const EpiArgs& ea, SlabEpi* se) {
  if (ea.s1 == 0.0 || ea.keep_half >= 0) return false;
  *se = SlabEpi{};
  se->nv = 0;
  const double gl = ea.wilson ? 1.0 : -1.0;
  for (int j = 0; j < 3; ++j) {
    if (ea.v[j] == nullptr) continue;
    const double c = -2.0 * ea.w[j] / ea.s1;
    se->v[se->nv] = ea.v[j];
    se->vcu[se->nv] = (float)c;
    se->vcl[se->nv] = (float)(gl * c);
    ++se->nv;
  }
  se->xs2 = (float)(-2.0 * (ea.wilson ? 4.0 : 4.0 - ea.m_w));
  se->fs = (float)(-0.5 * ea.s1);
  se->kgamma = ea.wilson ? 0 : 1;
  se->z = ea.z;
  se->wz = (float)ea.wz;
  se->g5_out = ea.g5_out;
  se->y = ea.y;
  se->c0 = (float)ea.c0;
  return true;
}

// Phases of one item: 0 XY, 1 Z+, 2 Z-, 3 T+, 4 T-, then 5 (v_0, v_1) and 6 (v_2) as needed.
__host__ __device__ inline int slab_phases(int nv) { return 5 + (nv + 1) / 2; }

// Grid: persistent CTAs of Lx Ly compute threads + one producer warp over the
// work items (rhs, slice), item = blockIdx.x + k gridDim.x, slice = z + Lz t;
// step j of a CTA is phase j % nph of its item j / nph and uses slot j % S.
// T: storage of links, input and v_j; OT: storage of z, y and the output.
template <class T, class OT>
__global__ void __launch_bounds__(kSlabMaxThreads, 1)
    k_dslash_slab(Geo g, const char* __restrict__ links, const char* __restrict__ in, char* out, SlabEpi e,
                  long long rhs_bytes, long long out_rhs_bytes, int nrhs, int nslots, volatile int* err,
                  const int* stall, long long stall_cycles) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int P = g.LxLy;
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  const int V = g.V;
  const uint32_t spb = (uint32_t)P * 16, lkb = (uint32_t)P * 8;  // bytes of one chunk of a plane
  const size_t slotb = (size_t)3 * spb + (size_t)6 * lkb;      // = two spinor planes
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + (size_t)nslots * slotb);
  unsigned long long* empty = full + kSlabMaxSlots;
  const int tid = threadIdx.x;
  const int nwarps = P / 32;  // compute warps
  const int nslices = Lz * Lt;
  const int nph = slab_phases(e.nv);
  const long long nitems = (long long)nslices * nrhs;
  const long long my_items = ((long long)blockIdx.x < nitems) ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long nsteps = my_items * nph;

  if (tid == 0) {
    for (int k = 0; k < nslots; ++k) {
      mbar_init(smem_u32(&full[k]), 1);
      mbar_init(smem_u32(&empty[k]), nwarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= P) {  // ---- producer warp: lane 0 issues every copy
    if (tid != P) return;
    long long j = 0, round = 0;
    int slot = 0, q = 0;
    long long item = blockIdx.x;
    bool ok = true;
    for (; j < nsteps; ++j) {
      if (round > 0 && !mbar_wait(smem_u32(&empty[slot]), (uint32_t)((round - 1) & 1), stall, stall_cycles)) {
        ok = false;
        break;
      }
      const int rhs = (int)(item / nslices), slice = (int)(item % nslices);
      unsigned char* buf = smem + (size_t)slot * slotb;
      const uint32_t bar = smem_u32(&full[slot]);
      const long long roff = (long long)rhs * rhs_bytes;
      if (q < 5) {
        const int t = slice / Lz, z = slice - t * Lz;
        int sp_slice = slice, lk_slice = slice, mu = 0;
        if (q == 1) {
          sp_slice = (z == Lz - 1) ? slice - (Lz - 1) : slice + 1;
          mu = 2;
        } else if (q == 2) {
          sp_slice = lk_slice = (z == 0) ? slice + (Lz - 1) : slice - 1;
          mu = 2;
        } else if (q == 3) {
          sp_slice = (t == Lt - 1) ? slice - (Lt - 1) * Lz : slice + Lz;
          mu = 3;
        } else if (q == 4) {
          sp_slice = lk_slice = (t == 0) ? slice + (Lt - 1) * Lz : slice - Lz;
          mu = 3;
        }
        const int nlk = (q == 0) ? 2 : 1;  // XY: U_x and U_y
        mbar_expect_tx(bar, 3 * spb + (uint32_t)nlk * 3 * lkb);
        for (int c = 0; c < 3; ++c)
          bulk_copy(smem_u32(buf + (size_t)c * spb), in + roff + ((long long)c * V + (long long)sp_slice * P) * 16,
                    spb, bar);
        for (int b = 0; b < nlk; ++b)
          for (int c = 0; c < 3; ++c)
            bulk_copy(smem_u32(buf + (size_t)3 * spb + ((size_t)b * 3 + c) * lkb),
                      links + ((long long)((mu + b) * 3 + c) * V + (long long)lk_slice * P) * 8,
                      lkb, bar);
      } else {  // planes of v_{2(q-5)} and v_{2(q-5)+1}
        const int v0 = 2 * (q - 5), nvp = min(2, e.nv - v0);
        mbar_expect_tx(bar, (uint32_t)nvp * 3 * spb);
        for (int b = 0; b < nvp; ++b) {
          const int jv = v0 + b;  // constant-index selects keep the parameter struct out of local memory
          const void* vp = (jv == 0) ? e.v[0] : (jv == 1) ? e.v[1] : e.v[2];
          const char* vb = static_cast<const char*>(vp) + roff;
          for (int c = 0; c < 3; ++c)
            bulk_copy(smem_u32(buf + ((size_t)b * 3 + c) * spb), vb + ((long long)c * V + (long long)slice * P) * 16,
                      spb, bar);
        }
      }
      if (++slot == nslots) {
        slot = 0;
        ++round;
      }
      if (++q == nph) {
        q = 0;
        item += gridDim.x;
      }
    }
    if (!ok) *err = 1;
    // let every copy issued land before the CTA can exit: the last use of each slot
    for (long long k = (j > nslots ? j - nslots : 0); k < j; ++k)
      mbar_wait(smem_u32(&full[k % nslots]), (uint32_t)((k / nslots) & 1));
    return;
  }

  // ---- compute warps
  const int lane = tid & 31;
  const int y = tid / Lx, x = tid - y * Lx;
  const int xp = (x == Lx - 1) ? tid - (Lx - 1) : tid + 1;
  const int xm = (x == 0) ? tid + (Lx - 1) : tid - 1;
  const int yp = (y == Ly - 1) ? tid - (Ly - 1) * Lx : tid + Lx;
  const int ym = (y == 0) ? tid + (Ly - 1) * Lx : tid - Lx;
  int slot = 0, q = 0;
  uint32_t par = 0;
  long long item = blockIdx.x;
  Spinor<float> acc;
  for (long long j = 0; j < nsteps; ++j) {
    if (!mbar_wait(smem_u32(&full[slot]), par, stall, stall_cycles)) {
      *err = 1;
      return;
    }
    const unsigned char* sp = smem + (size_t)slot * slotb;
    const unsigned char* lk0 = sp + (size_t)3 * spb;  // also the second spinor plane of a v phase
    if (q == 0) {
      const unsigned char* lk1 = lk0 + (size_t)3 * lkb;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc.c[k] = {0.f, 0.f};
      slab_axpy<T>(sp, P, tid, e.xs2, e.xs2, acc);
      slab_hop<0, -1, T>(sp, lk0, P, xp, tid, false, acc);
      slab_hop<0, +1, T>(sp, lk0, P, xm, xm, false, acc);
      slab_hop<1, -1, T>(sp, lk1, P, yp, tid, false, acc);
      slab_hop<1, +1, T>(sp, lk1, P, ym, ym, false, acc);
    } else if (q == 1) {
      slab_hop<2, -1, T>(sp, lk0, P, tid, tid, false, acc);
    } else if (q == 2) {
      slab_hop<2, +1, T>(sp, lk0, P, tid, tid, false, acc);
    } else if (q < 5) {
      const int t = (int)(item % nslices) / Lz;
      if (q == 3) slab_hop<3, -1, T>(sp, lk0, P, tid, tid, g.antiperiodic_t && t == Lt - 1, acc);
      else slab_hop<3, +1, T>(sp, lk0, P, tid, tid, g.antiperiodic_t && t == 0, acc);
    } else {
      if (q == 5) {
        slab_axpy<T>(sp, P, tid, e.vcu[0], e.vcl[0], acc);
        if (e.nv > 1) slab_axpy<T>(lk0, P, tid, e.vcu[1], e.vcl[1], acc);
      } else {
        slab_axpy<T>(sp, P, tid, e.vcu[2], e.vcl[2], acc);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&empty[slot]));  // this warp is done with the slot
    if (q == nph - 1) {
      const int rhs = (int)(item / nslices), slice = (int)(item % nslices);
      const int s = slice * P + tid;
      const long long ooff = (long long)rhs * out_rhs_bytes;
      Spinor<float> r;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float f = (e.kgamma && k >= 6) ? -e.fs : e.fs;
        r.c[k] = f * acc.c[k];
      }
      if (e.z != nullptr) {
        Spinor<float> zv;
        load_spinor_as<OT, float>(static_cast<const char*>(e.z) + ooff, s, V, zv);
#pragma unroll
        for (int k = 0; k < 12; ++k) r.c[k] = r.c[k] + e.wz * zv.c[k];
      }
      if (e.g5_out) {
#pragma unroll
        for (int k = 6; k < 12; ++k) r.c[k] = -1.f * r.c[k];
      }
      if (e.y != nullptr) {
        Spinor<float> yv;
        load_spinor_as<OT, float>(static_cast<const char*>(e.y) + ooff, s, V, yv);
#pragma unroll
        for (int k = 0; k < 12; ++k) r.c[k] = r.c[k] + e.c0 * yv.c[k];
      }
      store_spinor_as<OT, float>(out + ooff, s, V, r);
    }
    if (++slot == nslots) {
      slot = 0;
      par ^= 1;
    }
    if (++q == nph) {
      q = 0;
      item += gridDim.x;
    }
  }
}

}  // namespace slab

// Lattices the slab kernel takes: a whole (x, y) plane per CTA (a multiple of
// 32 sites, the producer warp on top at most kSlabMaxThreads), at least two
// slots in shared memory, even V (16-byte aligned chunks).
inline bool slab_supported(const LatticeH& g) {
  const int P = g.L[0] * g.L[1];
  return P % 32 == 0 && P + 32 <= slab::kSlabMaxThreads && slab::slab_slots(P) >= 2 && g.V % 2 == 0;
}

// Returns false (nothing launched) when the lattice, the epilogue (s1 = 0) or
// a pointer does not meet the kernel's requirements.
template <class T, class OT>
bool launch_slab(const DslashCfg& c, const LatticeH& gh, const void* links, const void* in, void* out,
                 const EpiArgs& ea, int nrhs, cudaStream_t st) {
  if (!slab_supported(gh) || c.err == nullptr || c.slab <= 0) return false;
  slab::SlabEpi se;
  if (!slab::slab_epi(ea, &se)) return false;
  uintptr_t al = reinterpret_cast<uintptr_t>(links) | reinterpret_cast<uintptr_t>(in);
  for (int j = 0; j < se.nv; ++j) al |= reinterpret_cast<uintptr_t>(se.v[j]);
  if (al & 15) return false;
  const Geo g = make_geo(gh);
  const int P = g.LxLy;
  const size_t smem = slab::slab_smem_bytes(P);
  if (cudaFuncSetAttribute(slab::k_dslash_slab<T, OT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return false;
  const long long rb = (long long)Store<T>::bytes_per_site * g.V, orb = (long long)Store<OT>::bytes_per_site * g.V;
  const long long nitems = (long long)gh.L[2] * gh.L[3] * nrhs;
  const unsigned grid = (unsigned)std::min<long long>(nitems, c.slab);
  launch_windowed(slab::k_dslash_slab<T, OT>, dim3(grid), dim3(P + 32), smem, st, links, false, g,
                  static_cast<const char*>(links), static_cast<const char*>(in), static_cast<char*>(out), se, rb, orb,
                  nrhs, slab::slab_slots(P), static_cast<volatile int*>(c.err), c.stall, c.stall_cycles);
  return true;
}

}  // namespace ov
