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
    k_force_pairs<F64><<<grid, 128, 0, st>>>(g, links, P, G);
  } else {
    PairArgsDev<float> P;
    args(&P);
    k_force_pairs<F32><<<grid, 128, 0, st>>>(g, links, P, G);
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
