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

__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// out = U in (each of the two spin components), complex products as FMA chains.
template <class R>
__device__ __forceinline__ void mul_u(const SU3<R>& u, const Half<R>& in, Half<R>& out) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx<R> u0 = u.u[3 * a], u1 = u.u[3 * a + 1], u2 = u.u[3 * a + 2];
      const cplx<R> h0 = in.c[3 * sp], h1 = in.c[3 * sp + 1], h2 = in.c[3 * sp + 2];
      R re = u0.re * h0.re;
      re = fma_(-u0.im, h0.im, re);
      re = fma_(u1.re, h1.re, re);
      re = fma_(-u1.im, h1.im, re);
      re = fma_(u2.re, h2.re, re);
      re = fma_(-u2.im, h2.im, re);
      R im = u0.re * h0.im;
      im = fma_(u0.im, h0.re, im);
      im = fma_(u1.re, h1.im, im);
      im = fma_(u1.im, h1.re, im);
      im = fma_(u2.re, h2.im, im);
      im = fma_(u2.im, h2.re, im);
      out.c[3 * sp + a] = {re, im};
    }
}

// out = U^dagger in:  out_a = sum_b conj(U_ba) in_b.
template <class R>
__device__ __forceinline__ void mul_udag(const SU3<R>& u, const Half<R>& in, Half<R>& out) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx<R> u0 = u.u[a], u1 = u.u[3 + a], u2 = u.u[6 + a];
      const cplx<R> h0 = in.c[3 * sp], h1 = in.c[3 * sp + 1], h2 = in.c[3 * sp + 2];
      R re = u0.re * h0.re;
      re = fma_(u0.im, h0.im, re);
      re = fma_(u1.re, h1.re, re);
      re = fma_(u1.im, h1.im, re);
      re = fma_(u2.re, h2.re, re);
      re = fma_(u2.im, h2.im, re);
      R im = u0.re * h0.im;
      im = fma_(-u0.im, h0.re, im);
      im = fma_(u1.re, h1.im, im);
      im = fma_(-u1.im, h1.re, im);
      im = fma_(u2.re, h2.im, im);
      im = fma_(-u2.im, h2.re, im);
      out.c[3 * sp + a] = {re, im};
    }
}

template <class R>
__device__ __forceinline__ void scale_half(Half<R>& h, R s) {
#pragma unroll
  for (int k = 0; k < 6; ++k) h.c[k] = s * h.c[k];
}


// --- 16-bit storage: projection in packed half2 arithmetic -----------------
// The neighbour spinor is loaded as 12 packed (re, im) 16-bit pairs and the
// two-spinor h = (p0 -/+ ..., p1 -/+ ...) is formed with packed additions on
// the stored values; only the 6 components of h are converted to FP32.  All
// products and accumulations stay in FP32.

template <class T> struct Pk;
template <> struct Pk<F16> {
  using H2 = __half2;
  __device__ static H2 from(uint32_t w) { return *reinterpret_cast<H2*>(&w); }
  __device__ static float2 to_f2(H2 h) { return __half22float2(h); }
  __device__ static H2 pm() { return __floats2half2_rn(-1.f, 1.f); }  // multiplies (swap) for +i
  __device__ static H2 mp() { return __floats2half2_rn(1.f, -1.f); }  // and for -i
};
template <> struct Pk<B16> {
  using H2 = __nv_bfloat162;
  __device__ static H2 from(uint32_t w) { return *reinterpret_cast<H2*>(&w); }
  __device__ static float2 to_f2(H2 h) { return __bfloat1622float2(h); }
  __device__ static H2 pm() { return __floats2bfloat162_rn(-1.f, 1.f); }
  __device__ static H2 mp() { return __floats2bfloat162_rn(1.f, -1.f); }
};

// p + i q  and  p - i q  on packed (re, im) pairs
template <class T>
__device__ __forceinline__ typename Pk<T>::H2 add_i(typename Pk<T>::H2 p, typename Pk<T>::H2 q) {
  return __hfma2(__lowhigh2highlow(q), Pk<T>::pm(), p);
}
template <class T>
__device__ __forceinline__ typename Pk<T>::H2 sub_i(typename Pk<T>::H2 p, typename Pk<T>::H2 q) {
  return __hfma2(__lowhigh2highlow(q), Pk<T>::mp(), p);
}

template <int MU, int SIGN, class T>
__device__ __forceinline__ void project16(const uint32_t (&w)[12], Half<float>& h) {
  using H2 = typename Pk<T>::H2;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const H2 p0 = Pk<T>::from(w[a]), p1 = Pk<T>::from(w[3 + a]), p2 = Pk<T>::from(w[6 + a]),
             p3 = Pk<T>::from(w[9 + a]);
    H2 h0, h1;
    if constexpr (MU == 0) {
      if constexpr (SIGN < 0) { h0 = sub_i<T>(p0, p3); h1 = sub_i<T>(p1, p2); }
      else                    { h0 = add_i<T>(p0, p3); h1 = add_i<T>(p1, p2); }
    } else if constexpr (MU == 1) {
      if constexpr (SIGN < 0) { h0 = __hadd2(p0, p3); h1 = __hsub2(p1, p2); }
      else                    { h0 = __hsub2(p0, p3); h1 = __hadd2(p1, p2); }
    } else if constexpr (MU == 2) {
      if constexpr (SIGN < 0) { h0 = sub_i<T>(p0, p2); h1 = add_i<T>(p1, p3); }
      else                    { h0 = add_i<T>(p0, p2); h1 = sub_i<T>(p1, p3); }
    } else {
      if constexpr (SIGN < 0) { h0 = __hsub2(p0, p2); h1 = __hsub2(p1, p3); }
      else                    { h0 = __hadd2(p0, p2); h1 = __hadd2(p1, p3); }
    }
    const float2 f0 = Pk<T>::to_f2(h0), f1 = Pk<T>::to_f2(h1);
    h.c[a] = {f0.x, f0.y};
    h.c[3 + a] = {f1.x, f1.y};
  }
}

// the 12 packed pairs of one site (spinor component k = 3*spin + colour in word k)
__device__ __forceinline__ void load_words16(const void* p, int s, int V, uint32_t (&w)[12]) {
  const uint4* q = static_cast<const uint4*>(p);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const uint4 v = __ldg(q + c * V + s);
    w[4 * c] = v.x;
    w[4 * c + 1] = v.y;
    w[4 * c + 2] = v.z;
    w[4 * c + 3] = v.w;
  }
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
