// Block kernels of the eigensolver that supplies the deflated eigenpairs of
// Eq. 3 (Sec. 2 precomputes them with a polynomial-preconditioned Lanczos;
// here: Chebyshev-filtered block subspace iteration with Rayleigh-Ritz):
//   * seeded Gaussian start vectors (counter-based hash, reproducible),
//   * Gram matrices G_ij = <A_i, B_j> of two blocks, FP64 sums,
//   * block rotation out_j = sum_i Y_i Q_ij.
#include "common.cuh"
#include "internal.h"

namespace ov {

// --- counter-based Gaussian numbers (splitmix64 finaliser + Box-Muller) ---
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <class T>
__global__ void k_random_block(char* out, int m, int64_t V, uint64_t seed) {
  using R = typename Store<T>::R;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int j = blockIdx.y;
  Spinor<R> x;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const uint64_t h = mix64(seed ^ mix64(((uint64_t)j * (uint64_t)V + (uint64_t)s) * 12u + k));
    const double u1 = ((h >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (double)(mix64(h) >> 11) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    x.c[k] = {R(r * cospi(2.0 * u2)), R(r * sinpi(2.0 * u2))};
  }
  store_spinor<T, R>(out + (int64_t)j * Store<T>::bytes_per_site * V, s, V, x);
}

void launch_random_block(OpPrec p, void* out, int m, int64_t V, uint64_t seed, cudaStream_t st) {
  dim3 grid((unsigned)((V + 255) / 256), m);
  if (p == OP_F64) k_random_block<F64><<<grid, 256, 0, st>>>(static_cast<char*>(out), m, V, seed);
  else k_random_block<F32><<<grid, 256, 0, st>>>(static_cast<char*>(out), m, V, seed);
}

// --- Gram matrix --------------------------------------------------------------
// Each CTA stages kGramSites sites of every vector of both blocks in shared
// memory (as complex in the arithmetic type; B optionally multiplied by
// gamma5), then each thread accumulates a
// 4 x 4 tile of (i, j) pairs.  Per-chunk sums in R, running sums in FP64.
constexpr int kGramSites = 8;
constexpr int kGramMax = 64;  // max vectors per block (per side)
// shared-memory row of one vector: kGramSites * 12 complex + 1 of padding, so
// that lanes reading consecutive vectors j hit consecutive banks
constexpr int kGramStride = kGramSites * 12 + 1;

template <class T>
__global__ void __launch_bounds__(256) k_gram(const char* __restrict__ A, int ma, const char* __restrict__ B, int mb,
                                              int64_t V, double2* __restrict__ partial, int g5b) {
  using R = typename Store<T>::R;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* sa = reinterpret_cast<cplx<R>*>(smem_raw);  // [ma][kGramStride]
  cplx<R>* sb = sa + (size_t)kGramMax * kGramStride;    // [mb][kGramStride]
  const int tid = threadIdx.x;
  const int ti = tid / 16, tj = tid % 16;  // 16 x 16 threads, pairs (ti + 16 a, tj + 16 b), a, b < 4
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);
  const int64_t vbytes = (int64_t)Store<T>::bytes_per_site * V;
  const int64_t nchunks = (V + kGramSites - 1) / kGramSites;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t s0 = ch * kGramSites;
    __syncthreads();
    // stage: one (vector, site) per thread-iteration
    for (int idx = tid; idx < (ma + mb) * kGramSites; idx += blockDim.x) {
      const int v = idx / kGramSites, ls = idx % kGramSites;
      const int64_t s = s0 + ls;
      Spinor<R> x;
      if (s < V) {
        const char* base = (v < ma) ? A + (int64_t)v * vbytes : B + (int64_t)(v - ma) * vbytes;
        load_spinor<T, R>(base, s, V, x);
        if (g5b && v >= ma) {
#pragma unroll
          for (int k = 6; k < 12; ++k) x.c[k] = R(-1) * x.c[k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) x.c[k] = {R(0), R(0)};
      }
      cplx<R>* dst = ((v < ma) ? sa + (size_t)v * kGramStride : sb + (size_t)(v - ma) * kGramStride) + ls * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) dst[k] = x.c[k];
    }
    __syncthreads();
    cplx<R> part[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) part[a][b] = {R(0), R(0)};
    for (int e = 0; e < kGramSites * 12; ++e) {
      cplx<R> av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = ti + 16 * a;
        av[a] = (i < ma) ? sa[(size_t)i * kGramStride + e] : cplx<R>{R(0), R(0)};
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = tj + 16 * b;
        bv[b] = (j < mb) ? sb[(size_t)j * kGramStride + e] : cplx<R>{R(0), R(0)};
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) part[a][b] = part[a][b] + cmulc(av[a], bv[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b].x += (double)part[a][b].re;
        acc[a][b].y += (double)part[a][b].im;
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ti + 16 * a, j = tj + 16 * b;
      if (i < ma && j < mb) partial[((int64_t)i * mb + j) * gridDim.x + blockIdx.x] = acc[a][b];
    }
}

size_t gram_smem_bytes(OpPrec p) {
  const size_t c = (p == OP_F64) ? 16 : 8;
  return 2 * (size_t)kGramMax * kGramStride * c;
}

int gram_max_vectors() { return kGramMax; }

cudaError_t launch_gram(OpPrec p, const void* A, int ma, const void* B, int mb, int64_t V, double2* partial,
                        int nblk, cudaStream_t st, int g5b) {
  const size_t sm = gram_smem_bytes(p);
  if (p == OP_F64) {
    cudaError_t e = cudaFuncSetAttribute(k_gram<F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gram<F64><<<nblk, 256, sm, st>>>(static_cast<const char*>(A), ma, static_cast<const char*>(B), mb, V, partial, g5b);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_gram<F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gram<F32><<<nblk, 256, sm, st>>>(static_cast<const char*>(A), ma, static_cast<const char*>(B), mb, V, partial, g5b);
  }
  return cudaGetLastError();
}

// --- rotation out_j = sum_i Y_i Q[i][j] ------------------------------------------
constexpr int kRotJ = 4;

template <class T>
__global__ void k_rotate(const char* __restrict__ Y, int m_in, const double2* __restrict__ Q, int m_out,
                         char* __restrict__ out, int64_t V) {
  using R = typename Store<T>::R;
  // block b: output tile b % ntj, site tile b / ntj, so that the blocks of one
  // site tile run together and read each input chunk through L2 once
  const int ntj = (m_out + kRotJ - 1) / kRotJ;
  const int64_t s = (int64_t)(blockIdx.x / ntj) * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int j0 = (int)(blockIdx.x % ntj) * kRotJ;
  const int64_t vbytes = (int64_t)Store<T>::bytes_per_site * V;
  Spinor<R> acc[kRotJ];
#pragma unroll
  for (int b = 0; b < kRotJ; ++b)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[b].c[k] = {R(0), R(0)};
  for (int i = 0; i < m_in; ++i) {
    Spinor<R> y;
    load_spinor<T, R>(Y + (int64_t)i * vbytes, s, V, y);
#pragma unroll
    for (int b = 0; b < kRotJ; ++b) {
      if (j0 + b < m_out) {
        const double2 q = Q[(int64_t)i * m_out + j0 + b];
        const cplx<R> qq = {R(q.x), R(q.y)};
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[b].c[k] = acc[b].c[k] + cmul(qq, y.c[k]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < kRotJ; ++b)
    if (j0 + b < m_out) store_spinor<T, R>(out + (int64_t)(j0 + b) * vbytes, s, V, acc[b]);
}

void launch_rotate(OpPrec p, const void* Y, int m_in, const double2* Q, int m_out, void* out, int64_t V,
                   cudaStream_t st) {
  const unsigned grid = (unsigned)(((V + 127) / 128) * ((m_out + kRotJ - 1) / kRotJ));
  if (p == OP_F64)
    k_rotate<F64><<<grid, 128, 0, st>>>(static_cast<const char*>(Y), m_in, Q, m_out, static_cast<char*>(out), V);
  else
    k_rotate<F32><<<grid, 128, 0, st>>>(static_cast<const char*>(Y), m_in, Q, m_out, static_cast<char*>(out), V);
}

}  // namespace ov
