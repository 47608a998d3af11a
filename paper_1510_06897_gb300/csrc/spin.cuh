// Spin projection (1 -/+ gamma_mu) to two-spinors and back, and SU(3)
// mat-vecs on two-spinors, chiral (DeGrand-Rossi) basis.  With h = (h0, h1)
// the projected two-spinor, the full spinors are
//   x:  (1-g) psi = (h0, h1,  i h1,  i h0), h = (p0 - i p3, p1 - i p2)
//       (1+g) psi = (h0, h1, -i h1, -i h0), h = (p0 + i p3, p1 + i p2)
//   y:  (1-g) psi = (h0, h1, -h1,  h0),     h = (p0 + p3, p1 - p2)
//       (1+g) psi = (h0, h1,  h1, -h0),     h = (p0 - p3, p1 + p2)
//   z:  (1-g) psi = (h0, h1,  i h0, -i h1), h = (p0 - i p2, p1 + i p3)
//       (1+g) psi = (h0, h1, -i h0,  i h1), h = (p0 + i p2, p1 - i p3)
//   t:  (1-g) psi = (h0, h1, -h0, -h1),     h = (p0 - p2, p1 - p3)
//       (1+g) psi = (h0, h1,  h0,  h1),     h = (p0 + p2, p1 + p3)
#pragma once
#include "common.cuh"

namespace ov {

// SIGN = -1 selects (1 - gamma_mu), +1 selects (1 + gamma_mu).
template <int MU, int SIGN, class R>
__device__ __forceinline__ void project(const Spinor<R>& p, Half<R>& h) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cplx<R> p0 = p.c[a], p1 = p.c[3 + a], p2 = p.c[6 + a], p3 = p.c[9 + a];
    if constexpr (MU == 0) {
      if constexpr (SIGN < 0) { h.c[a] = p0 + tmi(p3); h.c[3 + a] = p1 + tmi(p2); }
      else                    { h.c[a] = p0 + ti(p3);  h.c[3 + a] = p1 + ti(p2); }
    } else if constexpr (MU == 1) {
      if constexpr (SIGN < 0) { h.c[a] = p0 + p3; h.c[3 + a] = p1 - p2; }
      else                    { h.c[a] = p0 - p3; h.c[3 + a] = p1 + p2; }
    } else if constexpr (MU == 2) {
      if constexpr (SIGN < 0) { h.c[a] = p0 + tmi(p2); h.c[3 + a] = p1 + ti(p3); }
      else                    { h.c[a] = p0 + ti(p2);  h.c[3 + a] = p1 + tmi(p3); }
    } else {
      if constexpr (SIGN < 0) { h.c[a] = p0 - p2; h.c[3 + a] = p1 - p3; }
      else                    { h.c[a] = p0 + p2; h.c[3 + a] = p1 + p3; }
    }
  }
}

template <int MU, int SIGN, class R>
__device__ __forceinline__ void expand_add(Spinor<R>& acc, const Half<R>& h) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cplx<R> h0 = h.c[a], h1 = h.c[3 + a];
    acc.c[a] = acc.c[a] + h0;
    acc.c[3 + a] = acc.c[3 + a] + h1;
    if constexpr (MU == 0) {
      if constexpr (SIGN < 0) { acc.c[6 + a] = acc.c[6 + a] + ti(h1);  acc.c[9 + a] = acc.c[9 + a] + ti(h0); }
      else                    { acc.c[6 + a] = acc.c[6 + a] + tmi(h1); acc.c[9 + a] = acc.c[9 + a] + tmi(h0); }
    } else if constexpr (MU == 1) {
      if constexpr (SIGN < 0) { acc.c[6 + a] = acc.c[6 + a] - h1; acc.c[9 + a] = acc.c[9 + a] + h0; }
      else                    { acc.c[6 + a] = acc.c[6 + a] + h1; acc.c[9 + a] = acc.c[9 + a] - h0; }
    } else if constexpr (MU == 2) {
      if constexpr (SIGN < 0) { acc.c[6 + a] = acc.c[6 + a] + ti(h0);  acc.c[9 + a] = acc.c[9 + a] + tmi(h1); }
      else                    { acc.c[6 + a] = acc.c[6 + a] + tmi(h0); acc.c[9 + a] = acc.c[9 + a] + ti(h1); }
    } else {
      if constexpr (SIGN < 0) { acc.c[6 + a] = acc.c[6 + a] - h0; acc.c[9 + a] = acc.c[9 + a] - h1; }
      else                    { acc.c[6 + a] = acc.c[6 + a] + h0; acc.c[9 + a] = acc.c[9 + a] + h1; }
    }
  }
}

template <class R>
__device__ __forceinline__ void mul_u(const SU3<R>& u, const Half<R>& in, Half<R>& out) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      out.c[3 * sp + a] = cmul(u.u[3 * a], in.c[3 * sp]) + cmul(u.u[3 * a + 1], in.c[3 * sp + 1]) +
                          cmul(u.u[3 * a + 2], in.c[3 * sp + 2]);
}

template <class R>
__device__ __forceinline__ void mul_udag(const SU3<R>& u, const Half<R>& in, Half<R>& out) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      out.c[3 * sp + a] = cmulc(u.u[a], in.c[3 * sp]) + cmulc(u.u[3 + a], in.c[3 * sp + 1]) +
                          cmulc(u.u[6 + a], in.c[3 * sp + 2]);
}

template <class R>
__device__ __forceinline__ void scale_half(Half<R>& h, R s) {
#pragma unroll
  for (int k = 0; k < 6; ++k) h.c[k] = s * h.c[k];
}


// (1 -/+ gamma_mu) psi as a full spinor
template <int MU, int SIGN, class R>
__device__ __forceinline__ void project_full(const Spinor<R>& p, Spinor<R>& out) {
  Half<R> h;
  project<MU, SIGN>(p, h);
#pragma unroll
  for (int k = 0; k < 12; ++k) out.c[k] = {R(0), R(0)};
  expand_add<MU, SIGN>(out, h);
}

}  // namespace ov
