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

// expand_add for the t direction with a sign sg = +-1 on the hop (the
// antiperiodic wrap), as FMAs instead of additions: no branch.
template <int SIGN, class R>
__device__ __forceinline__ void expand_add_t(Spinor<R>& acc, const Half<R>& h, R sg);

__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

template <int SIGN, class R>
__device__ __forceinline__ void expand_add_t(Spinor<R>& acc, const Half<R>& h, R sg) {
  const R sl = (SIGN < 0) ? -sg : sg;  // (1 -/+ gamma_t): lower spins -/+ the upper ones
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cplx<R> h0 = h.c[a], h1 = h.c[3 + a];
    acc.c[a] = {fma_(sg, h0.re, acc.c[a].re), fma_(sg, h0.im, acc.c[a].im)};
    acc.c[3 + a] = {fma_(sg, h1.re, acc.c[3 + a].re), fma_(sg, h1.im, acc.c[3 + a].im)};
    acc.c[6 + a] = {fma_(sl, h0.re, acc.c[6 + a].re), fma_(sl, h0.im, acc.c[6 + a].im)};
    acc.c[9 + a] = {fma_(sl, h1.re, acc.c[9 + a].re), fma_(sl, h1.im, acc.c[9 + a].im)};
  }
}

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

// The two-spinor as 6 packed 16-bit (re, im) words: hw[a] = h0, hw[3 + a] = h1.
template <int MU, int SIGN, class T>
__device__ __forceinline__ void project16w(const uint32_t (&w)[12], uint32_t (&hw)[6]) {
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
    hw[a] = *reinterpret_cast<uint32_t*>(&h0);
    hw[3 + a] = *reinterpret_cast<uint32_t*>(&h1);
  }
}

template <int MU, int SIGN, class T>
__device__ __forceinline__ void project16(const uint32_t (&w)[12], Half<float>& h) {
  uint32_t hw[6];
  project16w<MU, SIGN, T>(w, hw);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 f = unpack2<T>(hw[k]);
    h.c[k] = {f.x, f.y};
  }
}

// --- 16-bit operands straight into FP32 FMAs ---------------------------------
// fmx<T, HA, HB>(a, b, c) = (float)a_HA * (float)b_HB + c with one rounding,
// where a_0 / a_1 is the low (real) / high (imaginary) half of the packed word
// a (fma.rn.f32.f16 / .bf16: no separate conversion instruction).  The
// product of two 16-bit values is exact in FP32, so this equals fmaf on the
// converted values.
template <class T, int HA, int HB>
__device__ __forceinline__ float fmx(uint32_t a, uint32_t b, float c) {
  float d;
#define OV_FMX_ASM(TY, SA, SB)                                                                      \
  asm("{\n .reg .b16 a0, a1, b0, b1;\n mov.b32 {a0, a1}, %1;\n mov.b32 {b0, b1}, %2;\n fma.rn.f32." TY \
      " %0, " SA ", " SB ", %3;\n}"                                                                    \
      : "=f"(d)                                                                                     \
      : "r"(a), "r"(b), "f"(c))
  if constexpr (std::is_same<T, F16>::value) {
    if constexpr (HA == 0 && HB == 0) OV_FMX_ASM("f16", "a0", "b0");
    else if constexpr (HA == 0) OV_FMX_ASM("f16", "a0", "b1");
    else if constexpr (HB == 0) OV_FMX_ASM("f16", "a1", "b0");
    else OV_FMX_ASM("f16", "a1", "b1");
  } else {
    if constexpr (HA == 0 && HB == 0) OV_FMX_ASM("bf16", "a0", "b0");
    else if constexpr (HA == 0) OV_FMX_ASM("bf16", "a0", "b1");
    else if constexpr (HB == 0) OV_FMX_ASM("bf16", "a1", "b0");
    else OV_FMX_ASM("bf16", "a1", "b1");
  }
#undef OV_FMX_ASM
  return d;
}

constexpr uint32_t kNegBoth = 0x80008000u;  // sign bits of both 16-bit halves
constexpr uint32_t kNegHi = 0x80000000u;    // of the imaginary half
constexpr uint32_t kNegLo = 0x00008000u;    // of the real half

// 16-bit link words uw[0..5] (rows 0, 1) -> row 2 = conj(row0 x row1) in
// uw[6..8], products and sums in FP32 (same chain order as reconstruct_row2),
// rounded to the storage type.
template <class T>
__device__ __forceinline__ void reconstruct16(uint32_t (&uw)[9]) {
  const uint32_t n0 = uw[0] ^ kNegBoth, n1 = uw[1] ^ kNegBoth, n2 = uw[2] ^ kNegBoth;
  // conj(a b - c d), a, c from row 0 (an, cn their negations), b, d from row 1
  auto cc = [](uint32_t a, uint32_t an, uint32_t b, uint32_t c, uint32_t cn, uint32_t d) {
    float re = fmx<T, 0, 0>(a, b, 0.f);
    re = fmx<T, 1, 1>(an, b, re);
    re = fmx<T, 0, 0>(cn, d, re);
    re = fmx<T, 1, 1>(c, d, re);
    float im = fmx<T, 0, 1>(c, d, 0.f);
    im = fmx<T, 1, 0>(c, d, im);
    im = fmx<T, 0, 1>(an, b, im);
    im = fmx<T, 1, 0>(an, b, im);
    return pack2<T>(re, im);
  };
  uw[6] = cc(uw[1], n1, uw[5], uw[2], n2, uw[4]);
  uw[7] = cc(uw[2], n2, uw[3], uw[0], n0, uw[5]);
  uw[8] = cc(uw[0], n0, uw[4], uw[1], n1, uw[3]);
}

// The 9 packed words of U_mu(s) for 16-bit links: 12 stored reals, 3 uint2
// chunks per direction at [(mu * 3 + c) V + s] (row 2 rebuilt by
// reconstruct16), or all 18 in 36 bytes: entries 0-3 and 4-7 as uint4 chunks
// at [mu V + s] and [(4 + mu) V + s], entry 8 as a word at [mu V + s] after
// the 8 V uint4 chunks (every chunk array starts 16-byte aligned).
template <class T, int LREC>
__device__ __forceinline__ void load_link_words16(const void* p, int mu, int s, int V, uint32_t (&uw)[9]) {
  if constexpr (LREC == 18) {
    const uint4* q = static_cast<const uint4*>(p);
    const uint4 a = __ldg(q + (int64_t)mu * V + s), b = __ldg(q + (int64_t)(4 + mu) * V + s);
    uw[0] = a.x;
    uw[1] = a.y;
    uw[2] = a.z;
    uw[3] = a.w;
    uw[4] = b.x;
    uw[5] = b.y;
    uw[6] = b.z;
    uw[7] = b.w;
    uw[8] = __ldg(reinterpret_cast<const uint32_t*>(q + (int64_t)8 * V) + (int64_t)mu * V + s);
  } else {
    const uint2* q = static_cast<const uint2*>(p) + (int64_t)mu * 3 * V;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint2 v = __ldg(q + c * V + s);
      uw[2 * c] = v.x;
      uw[2 * c + 1] = v.y;
    }
    reconstruct16<T>(uw);
  }
}

// out = U h for both spin components, U and h as packed 16-bit words
// (uw[3 a + b] = U_ab), FP32 FMA chains in the order of mul_u.
template <class T>
__device__ __forceinline__ void mul_u16(const uint32_t (&uw)[9], const uint32_t (&hw)[6], Half<float>& out) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const uint32_t h0 = hw[3 * sp], h1 = hw[3 * sp + 1], h2 = hw[3 * sp + 2];
    const uint32_t g0 = h0 ^ kNegHi, g1 = h1 ^ kNegHi, g2 = h2 ^ kNegHi;  // conj(h)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const uint32_t u0 = uw[3 * a], u1 = uw[3 * a + 1], u2 = uw[3 * a + 2];
      float re = fmx<T, 0, 0>(u0, h0, 0.f);
      re = fmx<T, 1, 1>(u0, g0, re);
      re = fmx<T, 0, 0>(u1, h1, re);
      re = fmx<T, 1, 1>(u1, g1, re);
      re = fmx<T, 0, 0>(u2, h2, re);
      re = fmx<T, 1, 1>(u2, g2, re);
      float im = fmx<T, 0, 1>(u0, h0, 0.f);
      im = fmx<T, 1, 0>(u0, h0, im);
      im = fmx<T, 0, 1>(u1, h1, im);
      im = fmx<T, 1, 0>(u1, h1, im);
      im = fmx<T, 0, 1>(u2, h2, im);
      im = fmx<T, 1, 0>(u2, h2, im);
      out.c[3 * sp + a] = {re, im};
    }
  }
}

// out = U^dagger h: out_a = sum_b conj(U_ba) h_b, order of mul_udag.
template <class T>
__device__ __forceinline__ void mul_udag16(const uint32_t (&uw)[9], const uint32_t (&hw)[6], Half<float>& out) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const uint32_t h0 = hw[3 * sp], h1 = hw[3 * sp + 1], h2 = hw[3 * sp + 2];
    const uint32_t g0 = h0 ^ kNegLo, g1 = h1 ^ kNegLo, g2 = h2 ^ kNegLo;  // (-re, im)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const uint32_t u0 = uw[a], u1 = uw[3 + a], u2 = uw[6 + a];
      float re = fmx<T, 0, 0>(u0, h0, 0.f);
      re = fmx<T, 1, 1>(u0, h0, re);
      re = fmx<T, 0, 0>(u1, h1, re);
      re = fmx<T, 1, 1>(u1, h1, re);
      re = fmx<T, 0, 0>(u2, h2, re);
      re = fmx<T, 1, 1>(u2, h2, re);
      float im = fmx<T, 0, 1>(u0, h0, 0.f);
      im = fmx<T, 1, 0>(u0, g0, im);
      im = fmx<T, 0, 1>(u1, h1, im);
      im = fmx<T, 1, 0>(u1, g1, im);
      im = fmx<T, 0, 1>(u2, h2, im);
      im = fmx<T, 1, 0>(u2, g2, im);
      out.c[3 * sp + a] = {re, im};
    }
  }
}

// acc += s h for (re, im) pairs as one packed FP32 instruction (s = +-1)
__device__ __forceinline__ void add2(cplx<float>& acc, const cplx<float>& h) {
  const float2 r = __fadd2_rn(make_float2(acc.re, acc.im), make_float2(h.re, h.im));
  acc = {r.x, r.y};
}
__device__ __forceinline__ void fma2(cplx<float>& acc, float2 s, const cplx<float>& h) {
  const float2 r = __ffma2_rn(s, make_float2(h.re, h.im), make_float2(acc.re, acc.im));
  acc = {r.x, r.y};
}

// expand_add / expand_add_t for FP32 accumulators with paired additions
// wherever the (re, im) order is kept (upper spins; lower spins of y and t).
template <int MU, int SIGN>
__device__ __forceinline__ void expand_add2(Spinor<float>& acc, const Half<float>& h) {
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cplx<float> h0 = h.c[a], h1 = h.c[3 + a];
    add2(acc.c[a], h0);
    add2(acc.c[3 + a], h1);
    if constexpr (MU == 0) {
      if constexpr (SIGN < 0) { acc.c[6 + a] = acc.c[6 + a] + ti(h1);  acc.c[9 + a] = acc.c[9 + a] + ti(h0); }
      else                    { acc.c[6 + a] = acc.c[6 + a] + tmi(h1); acc.c[9 + a] = acc.c[9 + a] + tmi(h0); }
    } else if constexpr (MU == 1) {
      if constexpr (SIGN < 0) { fma2(acc.c[6 + a], m1, h1); add2(acc.c[9 + a], h0); }
      else                    { add2(acc.c[6 + a], h1); fma2(acc.c[9 + a], m1, h0); }
    } else if constexpr (MU == 2) {
      if constexpr (SIGN < 0) { acc.c[6 + a] = acc.c[6 + a] + ti(h0);  acc.c[9 + a] = acc.c[9 + a] + tmi(h1); }
      else                    { acc.c[6 + a] = acc.c[6 + a] + tmi(h0); acc.c[9 + a] = acc.c[9 + a] + ti(h1); }
    } else {
      if constexpr (SIGN < 0) { fma2(acc.c[6 + a], m1, h0); fma2(acc.c[9 + a], m1, h1); }
      else                    { add2(acc.c[6 + a], h0); add2(acc.c[9 + a], h1); }
    }
  }
}

template <int SIGN>
__device__ __forceinline__ void expand_add_t2(Spinor<float>& acc, const Half<float>& h, float sg) {
  const float sl = (SIGN < 0) ? -sg : sg;
  const float2 su = make_float2(sg, sg), sv = make_float2(sl, sl);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fma2(acc.c[a], su, h.c[a]);
    fma2(acc.c[3 + a], su, h.c[3 + a]);
    fma2(acc.c[6 + a], sv, h.c[a]);
    fma2(acc.c[9 + a], sv, h.c[3 + a]);
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


}  // namespace ov
