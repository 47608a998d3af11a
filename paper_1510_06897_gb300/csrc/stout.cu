// Over-improved stout smearing of the gauge links (Sec. 3 prepares its
// ensembles with 3 steps at rho = 0.1, eps = -0.25; stout smearing of
// Morningstar and Peardon with the over-improved staple of Moran and
// Leinweber, both cited there).  One step, all links at once from the old
// field:
//   C_mu(x)  = rho sum_{nu != mu, +-} [ (5 - 2 eps)/3 plaquette staple
//                                       - (1 - eps)/12 (three rectangle staples) ]
//   Omega    = C_mu(x) U_mu(x)^dagger,  A = 1/2 (Omega - Omega^dagger) - 1/6 tr(Omega - Omega^dagger)
//   U'_mu(x) = exp(A) U_mu(x)                           (A = i Q, Q traceless Hermitian)
// A staple is the parallel transporter from x to x + mu^ along a closed
// path through the link; a step along -nu from y uses U_nu(y - nu^)^dagger.
// Per (nu, side) the plaquette path is (nu', mu, -nu') and the rectangles
// (nu', nu', mu, -nu', -nu'), (nu', mu, mu, -nu', -mu), (-mu, nu', mu, mu, -nu').
//
// Kernel: one thread per link (site, mu), FP64, links in the interface layout
// (complex128 [4][V][3][3], 144 contiguous bytes per link).  Each thread walks
// its 6 plaquette and 18 rectangle staples (102 link loads, L1/L2 resident
// neighbourhoods) and exponentiates A by scaling and squaring of a degree-16
// Taylor polynomial (||A / 2^s||_F <= 1/2, truncation below 1e-19).
// Compute-bound set-up kernel, not on the solver's hot path.
#include <cmath>
#include <string>

#include "../../include/overlap.h"
#include "common.cuh"
#include "internal.h"

namespace ov {
void set_thread_error(const std::string& msg);  // read back by ov_last_error(NULL)
}

namespace {

using ov::cplx;
using C = cplx<double>;

struct M3 {
  C e[9];
};

__device__ __forceinline__ M3 m_id() {
  M3 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.e[i] = {(i % 4 == 0) ? 1.0 : 0.0, 0.0};
  return r;
}

__device__ __forceinline__ M3 m_mul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C s = ov::cmul(a.e[3 * i], b.e[j]);
      s = s + ov::cmul(a.e[3 * i + 1], b.e[3 + j]);
      s = s + ov::cmul(a.e[3 * i + 2], b.e[6 + j]);
      r.e[3 * i + j] = s;
    }
  return r;
}

__device__ __forceinline__ M3 m_adj(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.e[3 * i + j] = ov::conj(a.e[3 * j + i]);
  return r;
}

struct Geo {
  int L[4];
  int64_t V;
};

__device__ __forceinline__ int64_t site_of(const Geo& g, const int p[4]) {
  return (((int64_t)p[3] * g.L[2] + p[2]) * g.L[1] + p[1]) * g.L[0] + p[0];
}

__device__ __forceinline__ M3 load_link(const double2* __restrict__ U, const Geo& g, int mu, int64_t s) {
  const double2* src = U + ((int64_t)mu * g.V + s) * 9;
  M3 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double2 v = __ldg(src + i);
    r.e[i] = {v.x, v.y};
  }
  return r;
}

// Transporter along n signed (1-based) directions starting at site x.
__device__ M3 transport(const double2* __restrict__ U, const Geo& g, const int x[4], const int* steps, int n) {
  int p[4] = {x[0], x[1], x[2], x[3]};
  M3 m = m_id();
  for (int k = 0; k < n; ++k) {
    const int d = steps[k];
    const int dir = (d > 0 ? d : -d) - 1;
    M3 l;
    if (d > 0) {
      l = load_link(U, g, dir, site_of(g, p));
      p[dir] = (p[dir] + 1 == g.L[dir]) ? 0 : p[dir] + 1;
    } else {
      p[dir] = (p[dir] == 0) ? g.L[dir] - 1 : p[dir] - 1;
      l = m_adj(load_link(U, g, dir, site_of(g, p)));
    }
    m = (k == 0) ? l : m_mul(m, l);
  }
  return m;
}

// exp(A) by scaling and squaring: Horner form of the degree-16 Taylor
// polynomial of A / 2^s with ||A / 2^s||_F <= 1/2, then s squarings.
__device__ M3 expm3(M3 a) {
  double nf = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) nf += a.e[i].re * a.e[i].re + a.e[i].im * a.e[i].im;
  nf = sqrt(nf);
  int s = 0;
  double sc = 1.0;
  while (nf * sc > 0.5 && s < 64) {
    sc *= 0.5;
    ++s;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) a.e[i] = sc * a.e[i];
  M3 t = m_id();
  for (int k = 16; k >= 1; --k) {  // t = 1 + a t / k
    M3 at = m_mul(a, t);
    const double inv = 1.0 / k;
#pragma unroll
    for (int i = 0; i < 9; ++i) t.e[i] = inv * at.e[i];
    t.e[0].re += 1.0;
    t.e[4].re += 1.0;
    t.e[8].re += 1.0;
  }
  for (int k = 0; k < s; ++k) t = m_mul(t, t);
  return t;
}

__global__ void __launch_bounds__(128) k_stout_step(const double2* __restrict__ U, double2* __restrict__ out, Geo g,
                                                    double rho, double wp, double wr) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= 4 * g.V) return;
  const int mu = (int)(tid / g.V);
  const int64_t s = tid - (int64_t)mu * g.V;
  int x[4];
  {
    int64_t r = s;
    x[0] = (int)(r % g.L[0]);
    r /= g.L[0];
    x[1] = (int)(r % g.L[1]);
    r /= g.L[1];
    x[2] = (int)(r % g.L[2]);
    x[3] = (int)(r / g.L[2]);
  }
  const int m = mu + 1;
  M3 c;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = {0.0, 0.0};
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    for (int side = 0; side < 2; ++side) {
      const int n = side == 0 ? nu + 1 : -(nu + 1);
      const int plaq[3] = {n, m, -n};
      M3 p = transport(U, g, x, plaq, 3);
#pragma unroll
      for (int i = 0; i < 9; ++i) c.e[i] = c.e[i] + wp * p.e[i];
      if (wr != 0.0) {
        const int rect[3][5] = {{n, n, m, -n, -n}, {n, m, m, -n, -m}, {-m, n, m, m, -n}};
        for (int q = 0; q < 3; ++q) {
          M3 r = transport(U, g, x, rect[q], 5);
#pragma unroll
          for (int i = 0; i < 9; ++i) c.e[i] = c.e[i] + wr * r.e[i];
        }
      }
    }
  }
  const M3 u = load_link(U, g, mu, s);
  M3 om = m_mul(c, m_adj(u));
  M3 a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a.e[3 * i + j] = (0.5 * rho) * (om.e[3 * i + j] - ov::conj(om.e[3 * j + i]));
  const C tr3 = (1.0 / 3.0) * (a.e[0] + a.e[4] + a.e[8]);
  a.e[0] = a.e[0] - tr3;
  a.e[4] = a.e[4] - tr3;
  a.e[8] = a.e[8] - tr3;
  const M3 un = m_mul(expm3(a), u);
  double2* dst = out + ((int64_t)mu * g.V + s) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) dst[i] = make_double2(un.e[i].re, un.e[i].im);
}

ov_status smear_fail(ov_status s, const std::string& msg) {
  ov::set_thread_error(msg);
  return s;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" ov_status ov_stout_smear(const int dims[4], const void* links_in, void* links_out, double rho,
                                    double epsilon, int steps, void* cuda_stream) {
  ov::set_thread_error("");
  if (!dims || !links_in || !links_out) return smear_fail(OV_ERR_INVALID, "null argument");
  Geo g;
  g.V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2) return smear_fail(OV_ERR_INVALID, "every lattice extent must be >= 2");
    g.L[i] = dims[i];
    g.V *= dims[i];
    if (g.V > (1LL << 27)) return smear_fail(OV_ERR_INVALID, "lattice larger than 2^27 sites");
  }
  if (steps < 0 || !std::isfinite(rho) || !std::isfinite(epsilon))
    return smear_fail(OV_ERR_INVALID, "need steps >= 0 and finite rho, epsilon");
  if (!on_device(links_in) || !on_device(links_out))
    return smear_fail(OV_ERR_INVALID, "links_in and links_out must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t bytes = (size_t)4 * (size_t)g.V * 9 * sizeof(double2);
  const double wp = (5.0 - 2.0 * epsilon) / 3.0, wr = -(1.0 - epsilon) / 12.0;
  void* tmp[2] = {nullptr, nullptr};
  auto cleanup = [&]() {
    for (void*& t : tmp)
      if (t) {
        cudaFree(t);
        t = nullptr;
      }
  };
  const void* src = links_in;
  void* last = nullptr;
  for (int i = 0; i < steps; ++i) {
    void* dst = (i == steps - 1 && src != links_out) ? links_out : nullptr;
    if (!dst) {
      if (!tmp[i % 2]) {
        cudaError_t e = cudaMalloc(&tmp[i % 2], bytes);
        if (e != cudaSuccess) {
          cleanup();
          return smear_fail(e == cudaErrorMemoryAllocation ? OV_ERR_NOMEM : OV_ERR_CUDA,
                            std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
      }
      dst = tmp[i % 2];
    }
    const int64_t n = 4 * g.V;
    k_stout_step<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(static_cast<const double2*>(src),
                                                                static_cast<double2*>(dst), g, rho, wp, wr);
    src = dst;
    last = dst;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    if (steps == 0 && links_in != links_out)
      e = cudaMemcpyAsync(links_out, links_in, bytes, cudaMemcpyDeviceToDevice, st);
    else if (steps > 0 && last != links_out)
      e = cudaMemcpyAsync(links_out, last, bytes, cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return smear_fail(OV_ERR_CUDA, std::string("stout smearing: ") + cudaGetErrorString(e));
  return OV_OK;
}
