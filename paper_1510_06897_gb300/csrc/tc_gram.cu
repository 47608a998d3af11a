// Deflation projection for many right-hand sides on the 5th-generation tensor
// cores: C_ij = sum_k conj(phi_i[k]) (G psi_j)[k] (Eq. 3's phi_i^dagger psi,
// G = gamma5 for D^dagger), phi and psi FP32 vectors in the library's SoA
// layout (each vector a contiguous array of 24 V floats, (re, im) pairs).
//
// Real form: with a = phi_i and b = psi_j as interleaved (re, im) arrays,
//   Re C = sum a . b,   Im C = sum a . b~,   b~ = (b_im, -b_re) per pair,
// so one real GEMM D[128 x 32] = A[128 x K] B[32 x K]^T with A rows = phi_i
// (n_ev <= 128, zero rows above) and B rows = (b_j, b~_j) (2 nrhs <= 32)
// gives both.  Each FP32 operand is split into TF32 parts x = hi + lo and
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi (tcgen05.mma kind::tf32, FP32
// accumulators in tensor memory).  K is split over CTAs (one per SM); every
// kFlush chunks a CTA adds its tensor-memory accumulator into FP64 registers
// and restarts it, and at the end writes one FP64 partial per (i, j), which
// the fixed-order reduction of blas.cu sums.
//
// Pipeline per CTA (256 threads): all threads load a 64-float chunk of every
// row, split it and store it into one of two shared-memory stages in the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices); one
// thread issues the 24 MMAs of the chunk and commits them to the stage's
// mbarrier, so the next chunk is loaded while the tensor core works.  Every
// mbarrier wait is bounded (about a second); on expiry the kernel records an
// error flag, waits (bounded) for its own MMAs, frees its tensor memory and
// returns.
#include "common.cuh"
#include "internal.h"

namespace ov {

namespace {

constexpr int kTcM = 128;      // MMA M: rows of A (eigenvectors, zero padded)
constexpr int kTcN = 32;       // MMA N: 2 x right-hand sides (zero padded)
constexpr int kTcK = 64;       // floats per chunk and stage
constexpr int kTcThreads = 256;
constexpr int kFlush = 64;     // chunks per tensor-memory accumulation window
constexpr int kTmemCols = 32;

constexpr uint32_t kTileA = kTcM * kTcK * 4;  // bytes of one A part (hi or lo)
constexpr uint32_t kTileB = kTcN * kTcK * 4;
constexpr uint32_t kStage = 2 * kTileA + 2 * kTileB;  // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kSmemBytes = 2 * kStage + 1024;     // two stages + control block

// byte offset of element (row r, k) inside one part: core matrices of
// 8 rows x 16 bytes, 16 of them along K (64 floats) per 8-row group.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 16 + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start address, leading (K-direction)
// byte offset 128, stride (8-row direction) byte offset 2048, descriptor
// version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(2048 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, N = 32, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tc_load32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo with hi the TF32 truncation of x (low 13 mantissa bits cleared).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gram(const float* __restrict__ A, int ma, const float* __restrict__ B, int mb, long long K, int g5b,
              double2* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stage_base = smem;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + 2 * kStage);  // [0], [1]: stages
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + 2 * kStage + 64);
  int* timed_out_sm = reinterpret_cast<int*>(smem + 2 * kStage + 128);
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long half_k = K / 2;  // gamma5 flips the second half of each vector (spins 2, 3)

  // zero both stages once: rows >= ma / >= 2 mb and the K tail stay zero
  for (uint32_t i = tid; i < 2 * kStage / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(stage_base)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    *timed_out_sm = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  const long long nchunks = (K + kTcK - 1) / kTcK;
  double acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.0;
  int it = 0;           // chunks processed by this CTA
  int in_window = 0;    // chunks in the current accumulation window
  bool failed = false;
  int last_stage = -1;
  uint32_t last_parity = 0;

  auto flush = [&]() {
    // all MMAs issued so far are complete once the last commit's phase is
    if (last_stage >= 0) {
      const bool ok = mbar_wait(smem_u32(&bars[last_stage]), last_parity);
      if (__syncthreads_or(!ok)) failed = true;
    }
    tc_fence_after();
    if (!failed && warp < 4 && in_window > 0) {
      float v[32];
      tc_load32(tmem + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] += (double)v[i];
    }
    in_window = 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };

  for (long long ch = blockIdx.x; ch < nchunks && !failed; ch += gridDim.x) {
    const int stage = it & 1;
    const uint32_t use = (uint32_t)(it >> 1);
    unsigned char* st = stage_base + stage * kStage;
    if (use >= 1) {  // the MMAs that last read this stage must be complete
      const bool ok = mbar_wait(smem_u32(&bars[stage]), (use - 1) & 1);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    const long long k0 = ch * kTcK;
    // A rows.  Consecutive threads take consecutive rows (conflict-free
    // 16-byte shared stores); each thread moves one 32-byte sector (8 floats).
    for (int idx = tid; idx < ma * (kTcK / 8); idx += kTcThreads) {
      const int r = idx % ma, q8 = idx / ma;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kq = 8 * q8 + 4 * h;
        const long long k = k0 + kq;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < K) x = __ldg(reinterpret_cast<const float4*>(A + (long long)r * K + k));
        float4 hi, lo;
        split_tf32(x.x, hi.x, lo.x);
        split_tf32(x.y, hi.y, lo.y);
        split_tf32(x.z, hi.z, lo.z);
        split_tf32(x.w, hi.w, lo.w);
        const uint32_t off = tile_off(r, kq);
        *reinterpret_cast<float4*>(st + off) = hi;
        *reinterpret_cast<float4*>(st + kTileA + off) = lo;
      }
    }
    // B rows: b_j in row j, b~_j = (b_im, -b_re) pairs in row mb + j
    for (int idx = tid; idx < mb * (kTcK / 8); idx += kTcThreads) {
      const int j = idx % mb, q8 = idx / mb;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kq = 8 * q8 + 4 * h;
        const long long k = k0 + kq;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < K) {
          x = __ldg(reinterpret_cast<const float4*>(B + (long long)j * K + k));
          if (g5b && k >= half_k) x = make_float4(-x.x, -x.y, -x.z, -x.w);
        }
        const float4 xt = make_float4(x.y, -x.x, x.w, -x.z);
        float4 hi, lo, thi, tlo;
        split_tf32(x.x, hi.x, lo.x);
        split_tf32(x.y, hi.y, lo.y);
        split_tf32(x.z, hi.z, lo.z);
        split_tf32(x.w, hi.w, lo.w);
        split_tf32(xt.x, thi.x, tlo.x);
        split_tf32(xt.y, thi.y, tlo.y);
        split_tf32(xt.z, thi.z, tlo.z);
        split_tf32(xt.w, thi.w, tlo.w);
        const uint32_t off = tile_off(j, kq), offt = tile_off(mb + j, kq);
        *reinterpret_cast<float4*>(st + 2 * kTileA + off) = hi;
        *reinterpret_cast<float4*>(st + 2 * kTileA + kTileB + off) = lo;
        *reinterpret_cast<float4*>(st + 2 * kTileA + offt) = thi;
        *reinterpret_cast<float4*>(st + 2 * kTileA + kTileB + offt) = tlo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t a_hi = smem_u32(st), a_lo = a_hi + kTileA, b_hi = a_hi + 2 * kTileA, b_lo = b_hi + kTileB;
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint32_t koff = (uint32_t)kk * 256;  // 8 floats = two core matrices along K
        const uint32_t acc_in = (in_window > 0 || kk > 0) ? 1u : 0u;
        tc_mma(tmem, smem_desc(a_hi + koff), smem_desc(b_hi + koff), acc_in);
        tc_mma(tmem, smem_desc(a_hi + koff), smem_desc(b_lo + koff), 1u);
        tc_mma(tmem, smem_desc(a_lo + koff), smem_desc(b_hi + koff), 1u);
      }
      tc_commit(smem_u32(&bars[stage]));
    }
    last_stage = stage;
    last_parity = use & 1;
    ++it;
    ++in_window;
    if (in_window == kFlush) flush();
  }
  if (!failed) flush();
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    // bounded wait for this CTA's own MMAs before releasing tensor memory
    if (last_stage >= 0) mbar_wait(smem_u32(&bars[last_stage]), last_parity);
  }
  if (!failed && warp < 4) {
    const int row = tid;  // warps 0-3: lane quarter = rows 0..127
    if (row < ma) {
      for (int j = 0; j < mb; ++j)
        partial[((long long)row * mb + j) * gridDim.x + blockIdx.x] = make_double2(acc[j], acc[mb + j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

int tc_gram_max_rows() { return kTcM; }
int tc_gram_max_rhs() { return kTcN / 2; }

cudaError_t launch_tc_gram(const void* A, int ma, const void* B, int mb, int64_t V, int g5b, double2* partial,
                           int nblk, int* err, cudaStream_t st) {
  if (ma < 1 || ma > kTcM || mb < 1 || 2 * mb > kTcN) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  k_tc_gram<<<nblk, kTcThreads, kSmemBytes, st>>>(static_cast<const float*>(A), ma, static_cast<const float*>(B),
                                                  mb, 24LL * V, g5b, partial, err);
  return cudaGetLastError();
}

}  // namespace ov
