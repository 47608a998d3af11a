// Device-side types shared by the overlap kernels: complex arithmetic, the
// SoA storage formats of spinors and links in each precision, and lattice
// indexing.
//
// Site index s = ((t*Lz + z)*Ly + y)*Lx + x.  A spinor has 12 complex
// components k = 3*spin + colour.  Internal (SoA) storage, per right-hand side:
//   fp64 : 12 chunks of double2 (1 complex each),  chunk c of site s at [c*V + s]
//   fp32 :  6 chunks of float4  (2 complex each)
//   fp16 / bf16 : 3 chunks of uint4 (4 complex each, 8 halves)
// Links, direction mu, site s (the link s -> s+mu^):
//   fp64 : all 9 entries, 9 double2 at [(mu*9 + e)*V + s]
//   fp32 : rows 0 and 1 (reconstruct-12), 3 float4 at [(mu*3 + c)*V + s]
//   fp16 / bf16 : rows 0 and 1, 3 uint2 (2 complex each) at [(mu*3 + c)*V + s]
// Row 2 of a reconstruct-12 link is conj(row0 x row1), exact for SU(3).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace ov {

template <class R>
struct cplx {
  R re, im;
};

template <class R> __device__ __forceinline__ cplx<R> mk(R a, R b) { return {a, b}; }
template <class R> __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <class R> __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class R> __device__ __forceinline__ cplx<R> cmulc(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class R> __device__ __forceinline__ cplx<R> conj(cplx<R> a) { return {a.re, -a.im}; }
// i*a and -i*a
template <class R> __device__ __forceinline__ cplx<R> ti(cplx<R> a) { return {-a.im, a.re}; }
template <class R> __device__ __forceinline__ cplx<R> tmi(cplx<R> a) { return {a.im, -a.re}; }

template <class R>
struct Spinor {
  cplx<R> c[12];
};
template <class R>
struct Half {  // spin-projected two-spinor
  cplx<R> c[6];
};
template <class R>
struct SU3 {
  cplx<R> u[9];
};

// ---------------------------------------------------------------------------
// storage tags

struct F64 {};
struct F32 {};
struct F16 {};
struct B16 {};

template <class T> struct Store;

template <> struct Store<F64> {
  using R = double;
  static constexpr int chunks = 12;      // spinor chunks per site
  static constexpr int link_chunks = 9;  // link chunks per direction
  using chunk_t = double2;
  using link_chunk_t = double2;
  static constexpr int bytes_per_site = 192;
};
template <> struct Store<F32> {
  using R = float;
  static constexpr int chunks = 6;
  static constexpr int link_chunks = 3;
  using chunk_t = float4;
  using link_chunk_t = float4;
  static constexpr int bytes_per_site = 96;
};
template <> struct Store<F16> {
  using R = float;
  static constexpr int chunks = 3;
  static constexpr int link_chunks = 3;
  using chunk_t = uint4;
  using link_chunk_t = uint2;
  static constexpr int bytes_per_site = 48;
};
template <> struct Store<B16> {
  using R = float;
  static constexpr int chunks = 3;
  static constexpr int link_chunks = 3;
  using chunk_t = uint4;
  using link_chunk_t = uint2;
  static constexpr int bytes_per_site = 48;
};

// --- 16-bit pack helpers --------------------------------------------------
template <class T> __device__ __forceinline__ float2 unpack2(uint32_t w);
template <class T> __device__ __forceinline__ uint32_t pack2(float a, float b);

template <> __device__ __forceinline__ float2 unpack2<F16>(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
template <> __device__ __forceinline__ uint32_t pack2<F16>(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <> __device__ __forceinline__ float2 unpack2<B16>(uint32_t w) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
  return __bfloat1622float2(h);
}
template <> __device__ __forceinline__ uint32_t pack2<B16>(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ---------------------------------------------------------------------------
// spinor load / store (one site of one right-hand side; p points at chunk 0)

template <class T, class R>
__device__ __forceinline__ void load_spinor(const void* p, int s, int V, Spinor<R>& o);
template <class T, class R>
__device__ __forceinline__ void store_spinor(void* p, int s, int V, const Spinor<R>& o);

template <>
__device__ __forceinline__ void load_spinor<F64, double>(const void* p, int s, int V, Spinor<double>& o) {
  const double2* q = static_cast<const double2*>(p);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    double2 v = __ldg(q + c * V + s);
    o.c[c] = {v.x, v.y};
  }
}
template <>
__device__ __forceinline__ void store_spinor<F64, double>(void* p, int s, int V, const Spinor<double>& o) {
  double2* q = static_cast<double2*>(p);
#pragma unroll
  for (int c = 0; c < 12; ++c) q[c * V + s] = make_double2(o.c[c].re, o.c[c].im);
}
template <>
__device__ __forceinline__ void load_spinor<F32, float>(const void* p, int s, int V, Spinor<float>& o) {
  const float4* q = static_cast<const float4*>(p);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float4 v = __ldg(q + c * V + s);
    o.c[2 * c] = {v.x, v.y};
    o.c[2 * c + 1] = {v.z, v.w};
  }
}
template <>
__device__ __forceinline__ void store_spinor<F32, float>(void* p, int s, int V, const Spinor<float>& o) {
  float4* q = static_cast<float4*>(p);
#pragma unroll
  for (int c = 0; c < 6; ++c)
    q[c * V + s] = make_float4(o.c[2 * c].re, o.c[2 * c].im, o.c[2 * c + 1].re, o.c[2 * c + 1].im);
}
template <class T>
__device__ __forceinline__ void load_spinor16(const void* p, int s, int V, Spinor<float>& o) {
  const uint4* q = static_cast<const uint4*>(p);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uint4 v = __ldg(q + c * V + s);
    float2 a = unpack2<T>(v.x), b = unpack2<T>(v.y), d = unpack2<T>(v.z), e = unpack2<T>(v.w);
    o.c[4 * c] = {a.x, a.y};
    o.c[4 * c + 1] = {b.x, b.y};
    o.c[4 * c + 2] = {d.x, d.y};
    o.c[4 * c + 3] = {e.x, e.y};
  }
}
template <class T>
__device__ __forceinline__ void store_spinor16(void* p, int s, int V, const Spinor<float>& o) {
  uint4* q = static_cast<uint4*>(p);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uint4 v;
    v.x = pack2<T>(o.c[4 * c].re, o.c[4 * c].im);
    v.y = pack2<T>(o.c[4 * c + 1].re, o.c[4 * c + 1].im);
    v.z = pack2<T>(o.c[4 * c + 2].re, o.c[4 * c + 2].im);
    v.w = pack2<T>(o.c[4 * c + 3].re, o.c[4 * c + 3].im);
    q[c * V + s] = v;
  }
}
template <>
__device__ __forceinline__ void load_spinor<F16, float>(const void* p, int s, int V, Spinor<float>& o) {
  load_spinor16<F16>(p, s, V, o);
}
template <>
__device__ __forceinline__ void store_spinor<F16, float>(void* p, int s, int V, const Spinor<float>& o) {
  store_spinor16<F16>(p, s, V, o);
}
template <>
__device__ __forceinline__ void load_spinor<B16, float>(const void* p, int s, int V, Spinor<float>& o) {
  load_spinor16<B16>(p, s, V, o);
}
template <>
__device__ __forceinline__ void store_spinor<B16, float>(void* p, int s, int V, const Spinor<float>& o) {
  store_spinor16<B16>(p, s, V, o);
}

// Loading a spinor stored in type T into a different arithmetic type R.
template <class T, class R>
__device__ __forceinline__ void load_spinor_as(const void* p, int s, int V, Spinor<R>& o) {
  Spinor<typename Store<T>::R> tmp;
  load_spinor<T, typename Store<T>::R>(p, s, V, tmp);
#pragma unroll
  for (int k = 0; k < 12; ++k) o.c[k] = {R(tmp.c[k].re), R(tmp.c[k].im)};
}
template <class T, class R>
__device__ __forceinline__ void store_spinor_as(void* p, int s, int V, const Spinor<R>& o) {
  using RT = typename Store<T>::R;
  Spinor<RT> tmp;
#pragma unroll
  for (int k = 0; k < 12; ++k) tmp.c[k] = {RT(o.c[k].re), RT(o.c[k].im)};
  store_spinor<T, RT>(p, s, V, tmp);
}

// ---------------------------------------------------------------------------
// link load (direction mu, site s)

__device__ __forceinline__ float __fma_any(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double __fma_any(double a, double b, double c) { return __fma_rn(a, b, c); }

// conj(a b - c d) as FMA chains
template <class R>
__device__ __forceinline__ cplx<R> conj_cross(cplx<R> a, cplx<R> b, cplx<R> c, cplx<R> d) {
  R re = a.re * b.re;
  re = __fma_any(-a.im, b.im, re);
  re = __fma_any(-c.re, d.re, re);
  re = __fma_any(c.im, d.im, re);
  R im = c.re * d.im;
  im = __fma_any(c.im, d.re, im);
  im = __fma_any(-a.re, b.im, im);
  im = __fma_any(-a.im, b.re, im);
  return {re, im};
}

template <class R>
__device__ __forceinline__ void reconstruct_row2(SU3<R>& u) {
  // row2 = conj(row0 x row1)
  u.u[6] = conj_cross(u.u[1], u.u[5], u.u[2], u.u[4]);
  u.u[7] = conj_cross(u.u[2], u.u[3], u.u[0], u.u[5]);
  u.u[8] = conj_cross(u.u[0], u.u[4], u.u[1], u.u[3]);
}

template <class T, class R>
__device__ __forceinline__ void load_link(const void* p, int mu, int s, int V, SU3<R>& u);

template <>
__device__ __forceinline__ void load_link<F64, double>(const void* p, int mu, int s, int V, SU3<double>& u) {
  const double2* q = static_cast<const double2*>(p) + (int64_t)mu * 9 * V;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    double2 v = __ldg(q + e * V + s);
    u.u[e] = {v.x, v.y};
  }
}
template <>
__device__ __forceinline__ void load_link<F32, float>(const void* p, int mu, int s, int V, SU3<float>& u) {
  const float4* q = static_cast<const float4*>(p) + (int64_t)mu * 3 * V;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float4 v = __ldg(q + c * V + s);
    u.u[2 * c] = {v.x, v.y};
    u.u[2 * c + 1] = {v.z, v.w};
  }
  reconstruct_row2(u);
}

// ---------------------------------------------------------------------------
// lattice geometry

struct Lattice {
  int L[4];      // Lx, Ly, Lz, Lt
  int64_t V;
  int antiperiodic_t;
};

struct Coords {
  int x[4];
};

__device__ __forceinline__ Coords site_coords(const Lattice& g, int64_t s) {
  Coords c;
  int64_t r = s;
  c.x[0] = int(r % g.L[0]); r /= g.L[0];
  c.x[1] = int(r % g.L[1]); r /= g.L[1];
  c.x[2] = int(r % g.L[2]); r /= g.L[2];
  c.x[3] = int(r);
  return c;
}

// Neighbour of s in direction mu (dir = +1 / -1); stride[mu] = prod of L below mu.
__device__ __forceinline__ int64_t neighbour(const Lattice& g, const Coords& c, int64_t s, int mu, int dir,
                                             int64_t stride) {
  if (dir > 0) return (c.x[mu] == g.L[mu] - 1) ? s - (int64_t)(g.L[mu] - 1) * stride : s + stride;
  return (c.x[mu] == 0) ? s + (int64_t)(g.L[mu] - 1) * stride : s - stride;
}

}  // namespace ov
