// Link-derivative kernels for S = chi^dagger P(K) chi (undeflated polynomial
// of Eq. 3).  Only the hopping term of D_W (Eq. 2) depends on the links, so
// for a pair (u, v) with dS = w u^dagger dK v and dU_mu(x) = X U_mu(x):
//
//   u^dagger dK v = sum_{x,mu} tr(X G_mu(x)),
//   G_mu(x) = -1/2 U_mu(x) A + 1/2 B U_mu(x)^dagger,
//   A = sum_s v(x+mu^)_s [(1 - gamma_mu) gamma5 u(x)]_s^dagger,
//   B = sum_s v(x)_s     [(1 + gamma_mu) gamma5 u(x+mu^)]_s^dagger
//
// (colour outer products summed over spin).  k_force_pairs accumulates
// G_mu(x) over a batch of pairs with one read-modify-write of the
// accumulator per link; k_force_finish returns F = P_TA(G^dagger), the
// anti-Hermitian traceless matrix with dS/deps = sum Re tr(X^dagger F).
#include "common.cuh"
#include "internal.h"
#include "spin.cuh"

namespace ov {

template <class R>
struct PairArgsDev {
  const char* u[kMaxForcePairs];
  const char* v[kMaxForcePairs];
  R w[kMaxForcePairs];  // weights in the arithmetic type, converted on the host
  int n;
};

// M += sum_k a_k b_k^dagger over the two components of spin-projected
// two-spinors a, b (colour outer products).  With P = 1 -/+ gamma_mu,
// P^dagger P = 2 P and the lower spins of P x are unit-phase copies of its
// upper two (the projection table in spin.cuh), so
//   sum_s v_s [P a]_s^dagger = 1/2 sum_s [P v]_s [P a]_s^dagger
//                            = sum_{k=0,1} h_k(v) h_k(a)^dagger,
// h the two-spinor of project<MU, SIGN>: 18 complex products instead of 36.
template <class R>
__device__ __forceinline__ void outer_acc2(cplx<R> (&M)[9], const Half<R>& a, const Half<R>& b) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M[3 * i + j] = M[3 * i + j] + cmulc(b.c[3 * k + j], a.c[3 * k + i]);
}

template <int MU, class T, class R>
__device__ __forceinline__ void force_dir(const Lattice& g, const Coords& c, int64_t s, int64_t stride,
                                          const void* links, const PairArgsDev<R>& P, cplx<R>* G) {
  const int64_t V = g.V;
  const int64_t n = neighbour(g, c, s, MU, +1, stride);
  cplx<R> A[9], B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = B[k] = {R(0), R(0)};
  for (int p = 0; p < P.n; ++p) {
    const R w = P.w[p];
    Spinor<R> x;
    Half<R> hv, ha;
    // A += w v(x+mu) [(1 - g_mu) g5 u(x)]^dagger
    load_spinor<T, R>(P.u[p], s, V, x);
#pragma unroll
    for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
    project<MU, -1>(x, ha);
    load_spinor<T, R>(P.v[p], n, V, x);
    project<MU, -1>(x, hv);
    scale_half(hv, w);
    outer_acc2(A, hv, ha);
    // B += w v(x) [(1 + g_mu) g5 u(x+mu)]^dagger
    load_spinor<T, R>(P.u[p], n, V, x);
#pragma unroll
    for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
    project<MU, +1>(x, ha);
    load_spinor<T, R>(P.v[p], s, V, x);
    project<MU, +1>(x, hv);
    scale_half(hv, w);
    outer_acc2(B, hv, ha);
  }
  SU3<R> U;
  load_link<T, R>(links, MU, s, V, U);
  R sg = R(1);
  if (MU == 3 && g.antiperiodic_t && c.x[3] == g.L[3] - 1) sg = R(-1);
  // G += sg * (-1/2 U A + 1/2 B U^dagger)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<R> ua = {R(0), R(0)}, bu = {R(0), R(0)};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ua = ua + cmul(U.u[3 * i + k], A[3 * k + j]);
        bu = bu + cmul(B[3 * i + k], conj(U.u[3 * j + k]));
      }
      cplx<R>* gp = G + ((int64_t)(MU * 9 + 3 * i + j)) * V + s;
      *gp = *gp + (sg * R(0.5)) * (bu - ua);
    }
}

// A block is 32 consecutive sites x the 4 directions, warp mu taking
// direction mu: the four warps read the same u(x), v(x) of every pair at
// about the same time (one L2 read, three L1 hits), and the x neighbours are
// the next lane's own sites.
template <class T>
__global__ void __launch_bounds__(128) k_force_pairs(Lattice g, const void* __restrict__ links,
                                                     PairArgsDev<typename Store<T>::R> P, void* Gv) {
  using R = typename Store<T>::R;
  const int64_t s = blockIdx.x * (int64_t)32 + (threadIdx.x & 31);
  if (s >= g.V) return;
  cplx<R>* G = static_cast<cplx<R>*>(Gv);
  const Coords c = site_coords(g, s);
  const int64_t sy = g.L[0], sz = sy * g.L[1], st = sz * g.L[2];
  switch (threadIdx.x >> 5) {
    case 0: force_dir<0, T, R>(g, c, s, 1, links, P, G); break;
    case 1: force_dir<1, T, R>(g, c, s, sy, links, P, G); break;
    case 2: force_dir<2, T, R>(g, c, s, sz, links, P, G); break;
    default: force_dir<3, T, R>(g, c, s, st, links, P, G); break;
  }
}

template <int N>
__device__ __forceinline__ void cp_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory tiled form of the same sums.  A block covers a
// BX x BY x BZ x BT box of sites and thread (mu, i) the link (box site i, mu).
// For every pair, u and v over the box and its +x, +y, +z, +t faces are
// copied into shared memory once with cp.async, three stages deep (pairs
// p + 1 and p + 2 land while pair p is used; one barrier per pair), so each
// vector leaves L2 about
// (box + faces) / box times (2.6 for the FP32 box 8 x 2 x 2 x 2: rows of 8
// sites are whole 128-byte lines of each FP32 chunk array, and two 256-thread
// blocks fit on an SM) instead of once for the
// site and once more for every direction that reaches it from outside the
// block.  The pairs are folded in the same order with the same arithmetic as
// k_force_pairs.
template <class T, int BX, int BY, int BZ, int BT>
struct ForceTile {
  static constexpr int NB = BX * BY * BZ * BT;  // box sites; threads = 4 NB
  static constexpr int H0 = BY * BZ * BT, H1 = BX * BZ * BT, H2 = BX * BY * BT, H3 = BX * BY * BZ;
  static constexpr int NE = NB + H0 + H1 + H2 + H3;  // box + faces
  static constexpr int CH = std::is_same<T, F64>::value ? 12 : 6;  // 16-byte chunks per site
  static constexpr int STAGE = 2 * CH * NE * 16;                 // u and v of one pair
  static constexpr int NS = 3;                                   // stages
  static constexpr int SMEM = NS * STAGE + NE * 4;               // stages + site table
  static constexpr int NT = 4 * NB;                              // threads
  // two resident blocks per SM (<= 128 registers) when their shared memory fits
  static constexpr int MINB = (NT < 512 && 2 * (SMEM + 1024) <= 228 * 1024) ? 2 : 1;
  static constexpr int NI = (2 * CH * NE + NT - 1) / NT;         // copy items per thread and pair
  static bool fits(const LatticeH& g) {
    return g.L[0] % BX == 0 && g.L[1] % BY == 0 && g.L[2] % BZ == 0 && g.L[3] % BT == 0;
  }
};

// spinor of slot e of vector `which` (0: u, 1: v) of one stage
template <class T, class R, int NE, int CH>
__device__ __forceinline__ void smem_spinor(const unsigned char* stage, int which, int e, Spinor<R>& o) {
  if constexpr (CH == 12) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double2 v = *reinterpret_cast<const double2*>(stage + ((which * CH + c) * NE + e) * 16);
      o.c[c] = {R(v.x), R(v.y)};
    }
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(stage + ((which * CH + c) * NE + e) * 16);
      o.c[2 * c] = {R(v.x), R(v.y)};
      o.c[2 * c + 1] = {R(v.z), R(v.w)};
    }
  }
}

// one pair's contribution to A and B of link (box site i, MU); nb: slot of i + MU
template <int MU, class T, class R, class TG>
__device__ __forceinline__ void force_tile_pair(const unsigned char* st, int i, int nb, R w, cplx<R> (&A)[9],
                                                cplx<R> (&B)[9]) {
  Spinor<R> x;
  Half<R> hv, ha;
  // A += w v(x+mu) [(1 - g_mu) g5 u(x)]^dagger
  smem_spinor<T, R, TG::NE, TG::CH>(st, 0, i, x);
#pragma unroll
  for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
  project<MU, -1>(x, ha);
  smem_spinor<T, R, TG::NE, TG::CH>(st, 1, nb, x);
  project<MU, -1>(x, hv);
  scale_half(hv, w);
  outer_acc2(A, hv, ha);
  // B += w v(x) [(1 + g_mu) g5 u(x+mu)]^dagger
  smem_spinor<T, R, TG::NE, TG::CH>(st, 0, nb, x);
#pragma unroll
  for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
  project<MU, +1>(x, ha);
  smem_spinor<T, R, TG::NE, TG::CH>(st, 1, i, x);
  project<MU, +1>(x, hv);
  scale_half(hv, w);
  outer_acc2(B, hv, ha);
}

// G_MU(s) += sg (-1/2 U A + 1/2 B U^dagger)
template <int MU, class T, class R>
__device__ __forceinline__ void force_tile_store(const Lattice& g, const void* links, int64_t s, R sg,
                                                 const cplx<R> (&A)[9], const cplx<R> (&B)[9], cplx<R>* G) {
  const int64_t V = g.V;
  SU3<R> U;
  load_link<T, R>(links, MU, s, V, U);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<R> ua = {R(0), R(0)}, bu = {R(0), R(0)};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ua = ua + cmul(U.u[3 * a + k], A[3 * k + b]);
        bu = bu + cmul(B[3 * a + k], conj(U.u[3 * b + k]));
      }
      cplx<R>* gp = G + ((int64_t)(MU * 9 + 3 * a + b)) * V + s;
      *gp = *gp + (sg * R(0.5)) * (bu - ua);
    }
}

template <class T, int BX, int BY, int BZ, int BT>
__global__ void __launch_bounds__(ForceTile<T, BX, BY, BZ, BT>::NT, ForceTile<T, BX, BY, BZ, BT>::MINB)
    k_force_tile(Lattice g, const void* __restrict__ links, PairArgsDev<typename Store<T>::R> P, void* Gv) {
  using R = typename Store<T>::R;
  using TG = ForceTile<T, BX, BY, BZ, BT>;
  extern __shared__ __align__(16) unsigned char fsm[];
  int* ext = reinterpret_cast<int*>(fsm + TG::NS * TG::STAGE);
  const int tid = threadIdx.x;
  int b = blockIdx.x;
  const int nbx = g.L[0] / BX, nby = g.L[1] / BY, nbz = g.L[2] / BZ;
  const int X0 = (b % nbx) * BX;
  b /= nbx;
  const int Y0 = (b % nby) * BY;
  b /= nby;
  const int Z0 = (b % nbz) * BZ;
  const int T0 = (b / nbz) * BT;
  // lattice site of every slot: box sites, then the +x, +y, +z, +t faces
  for (int e = tid; e < TG::NE; e += TG::NT) {
    int c[4];
    if (e < TG::NB) {
      c[0] = e % BX;
      c[1] = (e / BX) % BY;
      c[2] = (e / (BX * BY)) % BZ;
      c[3] = e / (BX * BY * BZ);
    } else if (e < TG::NB + TG::H0) {
      const int f = e - TG::NB;
      c[0] = BX;
      c[1] = f % BY;
      c[2] = (f / BY) % BZ;
      c[3] = f / (BY * BZ);
    } else if (e < TG::NB + TG::H0 + TG::H1) {
      const int f = e - TG::NB - TG::H0;
      c[0] = f % BX;
      c[1] = BY;
      c[2] = (f / BX) % BZ;
      c[3] = f / (BX * BZ);
    } else if (e < TG::NB + TG::H0 + TG::H1 + TG::H2) {
      const int f = e - TG::NB - TG::H0 - TG::H1;
      c[0] = f % BX;
      c[1] = (f / BX) % BY;
      c[2] = BZ;
      c[3] = f / (BX * BY);
    } else {
      const int f = e - TG::NB - TG::H0 - TG::H1 - TG::H2;
      c[0] = f % BX;
      c[1] = (f / BX) % BY;
      c[2] = f / (BX * BY);
      c[3] = BT;
    }
    const int gx = (X0 + c[0]) % g.L[0], gy = (Y0 + c[1]) % g.L[1];
    const int gz = (Z0 + c[2]) % g.L[2], gt = (T0 + c[3]) % g.L[3];
    ext[e] = gx + g.L[0] * (gy + g.L[1] * (gz + g.L[2] * gt));
  }
  __syncthreads();
  // Copy items of this thread, the same for every pair: item idx = tid + m NT
  // is 16-byte chunk (idx / NE) % CH of slot idx % NE of u (idx < CH NE) or
  // v, which lands at byte 16 idx of the stage; its source is chunk-array
  // element ch V + site (< 12 * 2^27, 32 bits).
  uint32_t item[TG::NI];
#pragma unroll
  for (int m = 0; m < TG::NI; ++m) {
    const int idx = tid + m * TG::NT;
    item[m] = idx < 2 * TG::CH * TG::NE
                  ? (uint32_t)(((idx / TG::NE) % TG::CH) * g.V) + (uint32_t)ext[idx % TG::NE]
                  : 0u;
  }
  auto issue = [&](int p) {  // pair p's u and v into stage p % NS
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(fsm + (p % TG::NS) * TG::STAGE);
    const char* u = P.u[p];
    const char* v = P.v[p];
#pragma unroll
    for (int m = 0; m < TG::NI; ++m) {
      const int idx = tid + m * TG::NT;
      if (idx < 2 * TG::CH * TG::NE) {
        const char* src = (idx < TG::CH * TG::NE ? u : v) + (uint64_t)item[m] * 16u;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + (uint32_t)idx * 16u), "l"(src)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int mu = tid / TG::NB, i = tid % TG::NB;  // mu is warp-uniform: NB is a multiple of 32
  const int ix = i % BX, iy = (i / BX) % BY, iz = (i / (BX * BY)) % BZ, it = i / (BX * BY * BZ);
  int nb;  // slot of site i + mu
  if (mu == 0) nb = ix < BX - 1 ? i + 1 : TG::NB + (iy + BY * (iz + BZ * it));
  else if (mu == 1) nb = iy < BY - 1 ? i + BX : TG::NB + TG::H0 + (ix + BX * (iz + BZ * it));
  else if (mu == 2) nb = iz < BZ - 1 ? i + BX * BY : TG::NB + TG::H0 + TG::H1 + (ix + BX * (iy + BY * it));
  else nb = it < BT - 1 ? i + BX * BY * BZ : TG::NB + TG::H0 + TG::H1 + TG::H2 + (ix + BX * (iy + BY * iz));
  cplx<R> A[9], B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = B[k] = {R(0), R(0)};
  static_assert(TG::NS == 3, "the waits below assume three stages");
  if (P.n > 0) issue(0);
  if (P.n > 1) issue(1);
  for (int p = 0; p < P.n; ++p) {
    // groups committed so far: pairs 0 .. min(p + 1, n - 1); pair p must be complete
    if (p + 1 < P.n) cp_wait_group<1>();
    else cp_wait_group<0>();
    __syncthreads();  // every thread's copies of pair p have landed; pair p - 1 is used up
    if (p + 2 < P.n) issue(p + 2);  // into the stage of pair p - 1
    const unsigned char* st = fsm + (p % TG::NS) * TG::STAGE;
    const R w = P.w[p];
    switch (mu) {
      case 0: force_tile_pair<0, T, R, TG>(st, i, nb, w, A, B); break;
      case 1: force_tile_pair<1, T, R, TG>(st, i, nb, w, A, B); break;
      case 2: force_tile_pair<2, T, R, TG>(st, i, nb, w, A, B); break;
      default: force_tile_pair<3, T, R, TG>(st, i, nb, w, A, B); break;
    }
  }
  cplx<R>* G = static_cast<cplx<R>*>(Gv);
  const int64_t s = ext[i];
  const R sg = (mu == 3 && g.antiperiodic_t && T0 + it == g.L[3] - 1) ? R(-1) : R(1);
  switch (mu) {
    case 0: force_tile_store<0, T, R>(g, links, s, sg, A, B, G); break;
    case 1: force_tile_store<1, T, R>(g, links, s, sg, A, B, G); break;
    case 2: force_tile_store<2, T, R>(g, links, s, sg, A, B, G); break;
    default: force_tile_store<3, T, R>(g, links, s, sg, A, B, G); break;
  }
}

template <class T, int BX, int BY, int BZ, int BT>
void launch_force_tile(const Lattice& g, const void* links, const PairArgsDev<typename Store<T>::R>& P, void* G,
                       cudaStream_t st) {
  using TG = ForceTile<T, BX, BY, BZ, BT>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_force_tile<T, BX, BY, BZ, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TG::SMEM);
    attr = true;
  }
  k_force_tile<T, BX, BY, BZ, BT><<<(unsigned)(g.V / TG::NB), 4 * TG::NB, TG::SMEM, st>>>(g, links, P, G);
}

void launch_force_pairs(OpPrec p, const LatticeH& gh, const void* links, const ForcePairs& pairs, void* G,
                        cudaStream_t st) {
  Lattice g;
  for (int i = 0; i < 4; ++i) g.L[i] = gh.L[i];
  g.V = gh.V;
  g.antiperiodic_t = gh.antiperiodic_t;
  auto args = [&](auto* P) {
    P->n = pairs.n;
    for (int i = 0; i < pairs.n; ++i) {
      P->u[i] = static_cast<const char*>(pairs.u[i]);
      P->v[i] = static_cast<const char*>(pairs.v[i]);
      P->w[i] = static_cast<decltype(+P->w[0])>(pairs.w[i]);
    }
  };
  const unsigned grid = (unsigned)((g.V + 31) / 32);
  if (p == OP_F64) {
    PairArgsDev<double> P;
    args(&P);
    if (ForceTile<F64, 4, 4, 2, 2>::fits(gh)) launch_force_tile<F64, 4, 4, 2, 2>(g, links, P, G, st);
    else k_force_pairs<F64><<<grid, 128, 0, st>>>(g, links, P, G);
  } else {
    PairArgsDev<float> P;
    args(&P);
    if (ForceTile<F32, 8, 2, 2, 2>::fits(gh)) launch_force_tile<F32, 8, 2, 2, 2>(g, links, P, G, st);
    else k_force_pairs<F32><<<grid, 128, 0, st>>>(g, links, P, G);
  }
}

// F = P_TA(G^dagger) -> complex128 AoS [4][V][3][3]
template <class R>
__global__ void k_force_finish(const cplx<R>* __restrict__ G, int64_t V, double2* __restrict__ out) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int mu = blockIdx.y;
  double2 m[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const cplx<R> v = G[((int64_t)mu * 9 + e) * V + s];
    m[e] = make_double2((double)v.re, (double)v.im);
  }
  // H = G^dagger: H_ij = conj(G_ji); F = (H - H^dagger)/2 - tr(.)/3
  double2 f[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 hij = make_double2(m[3 * j + i].x, -m[3 * j + i].y);
      const double2 hji = make_double2(m[3 * i + j].x, -m[3 * i + j].y);
      f[3 * i + j] = make_double2(0.5 * (hij.x - hji.x), 0.5 * (hij.y + hji.y));
    }
  const double tr_im = (f[0].y + f[4].y + f[8].y) / 3.0;
  f[0].y -= tr_im;
  f[4].y -= tr_im;
  f[8].y -= tr_im;
  f[0].x = f[4].x = f[8].x = 0.0;
  double2* o = out + ((int64_t)mu * V + s) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) o[e] = f[e];
}

void launch_force_finish(OpPrec p, const void* G, int64_t V, void* out, cudaStream_t st) {
  dim3 grid((unsigned)((V + 255) / 256), 4);
  if (p == OP_F64)
    k_force_finish<double><<<grid, 256, 0, st>>>(static_cast<const cplx<double>*>(G), V, static_cast<double2*>(out));
  else
    k_force_finish<float><<<grid, 256, 0, st>>>(static_cast<const cplx<float>*>(G), V, static_cast<double2*>(out));
}

}  // namespace ov
