// Deflation projection for many right-hand sides on the 5th-generation tensor
// cores: C_ij = sum_k conj(phi_i[k]) (G psi_j)[k] (Eq. 3's phi_i^dagger psi,
// G = gamma5 for D^dagger), phi and psi FP32 vectors in the library's SoA
// layout (each vector a contiguous array of 24 V floats, (re, im) pairs).
//
// Real form: with a = phi_i and b = psi_j as interleaved (re, im) arrays,
//   Re C = sum a . b,   Im C = sum a . b~,   b~ = (b_im, -b_re) per pair.
// Each FP32 operand is split into TF32 parts x = hi + lo.  The B tile (the
// MMA's N side, 64 rows) holds b_j and b~_j as hi parts in rows 0 .. 2 mb - 1
// and as lo parts in rows 32 .. 32 + 2 mb - 1.  For n_ev <= 64 the A tile
// (M = 128) holds a_i hi in row i and a_i lo in row 64 + i, so ONE
// tcgen05.mma kind::tf32 per 8-wide K step yields all four products
// hi.hi, hi.lo (columns 0-31, 32-63 of lanes 0-63) and lo.hi, lo.lo (lanes
// 64-127); the lo.lo term is below the FP32 level but costs nothing.  For
// 64 < n_ev <= 128 the hi and lo parts of A sit in two 128-row tiles and two
// MMAs per K step accumulate into the same lanes.  FP32 accumulators live in
// tensor memory.  K is split over CTAs (one per SM); every kFlush chunks a
// CTA adds its tensor-memory accumulator into FP64 registers and restarts
// it, and at the end writes one FP64 partial per (i, j), which the
// fixed-order reduction of blas.cu sums.
//
// Pipeline per CTA (512 threads): raw 64-float chunks of every row are copied
// into a ring of up to four shared-memory buffers with cp.async (several
// chunks in flight), then split and stored into one of two MMA stages in the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices); one
// thread issues the chunk's 8 (or 16) MMAs and commits them to the stage's
// mbarrier, so the next chunk is loaded while the tensor core works.  Every
// mbarrier wait is bounded (about a second); on expiry the kernel records an
// error flag, waits (bounded) for its own MMAs, frees its tensor memory and
// returns.
#include "common.cuh"
#include "internal.h"

namespace ov {

namespace {

constexpr int kTcM = 128;      // MMA M: A tile rows
constexpr int kTcN = 64;       // MMA N: B tile rows (hi parts in 0..31, lo parts in 32..63)
constexpr int kLoRow = 32;     // first B row of the lo parts
constexpr int kPackRows = 64;  // n_ev <= 64: a_i lo in A row 64 + i
constexpr int kTcK = 64;       // floats per chunk and stage
constexpr int kTcThreads = 512;
constexpr int kRawPitch = kTcK * 4 + 16;  // bytes per raw row (padded: conflict-free 16-byte reads)
constexpr int kRawStagesMax = 4;          // chunks in flight (cp.async ring of raw FP32 rows)
constexpr int kFlush = 64;     // chunks per tensor-memory accumulation window
constexpr int kTmemCols = 64;

constexpr uint32_t kTileA = kTcM * kTcK * 4;  // bytes of one A tile
constexpr uint32_t kTileB = kTcN * kTcK * 4;
constexpr uint32_t kCtrl = 1024;                     // mbarriers, tensor-memory address
__host__ __device__ inline uint32_t stage_bytes(int ma) { return (ma <= kPackRows ? 1u : 2u) * kTileA + kTileB; }
// dynamic shared memory: two MMA stages, control block, raw ring
inline uint32_t raw_stages(int ma, int rows) {
  const uint32_t avail = 227u * 1024u - 2 * stage_bytes(ma) - kCtrl;
  const uint32_t per = (uint32_t)rows * kRawPitch;
  const uint32_t n = avail / per;
  return n < 1 ? 1 : (n > (uint32_t)kRawStagesMax ? (uint32_t)kRawStagesMax : n);
}

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

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, N = 64, M = 128.
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
// stall (testing, see ov_test_wait_expiry): a device flag that nothing sets;
// when given, the wait first waits up to stall_cycles for it, runs out and
// reports failure as an expired wait would.
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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gram(const float* __restrict__ A, int ma, const float* __restrict__ B, int mb, long long K, int g5b,
              double2* __restrict__ partial, int* __restrict__ err, int nraw, const int* stall,
              long long stall_cycles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const bool packed = ma <= kPackRows;
  const uint32_t kStage = stage_bytes(ma);
  const uint32_t offB = kStage - kTileB;  // B tile after the one or two A tiles
  unsigned char* stage_base = smem;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + 2 * kStage);  // [0], [1]: stages
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + 2 * kStage + 64);
  unsigned char* raw_base = smem + 2 * kStage + kCtrl;
  const int rows = ma + mb;
  const uint32_t raw_stage_bytes = (uint32_t)rows * kRawPitch;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long half_k = K / 2;  // gamma5 flips the second half of each vector (spins 2, 3)

  // zero both MMA stages once: rows no chunk writes stay zero
  for (uint32_t i = tid; i < 2 * kStage / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(stage_base)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
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
  // raw copy of chunk `chk` into ring slot `slot`: 16 bytes per thread-iteration,
  // zero-filled past K and for chunks past the end
  auto issue = [&](long long chk, int slot) {
    const uint32_t dst0 = smem_u32(raw_base + (uint32_t)slot * raw_stage_bytes);
    const long long k0 = chk * kTcK;
    for (int idx = tid; idx < rows * (kTcK / 4); idx += kTcThreads) {
      const int row = idx / (kTcK / 4), q = idx % (kTcK / 4);
      const long long k = k0 + 4 * q;
      const bool ok = chk < nchunks && k < K;
      const float* src = (row < ma) ? A + (long long)row * K : B + (long long)(row - ma) * K;
      cp_async16(dst0 + (uint32_t)row * kRawPitch + 16u * q, ok ? src + k : A, ok ? 16u : 0u);
    }
    cp_async_commit();
  };

  // FP64 sums of the hi-column (0..31) and lo-column (32..63) accumulators of this thread's lane
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
      const bool ok = mbar_wait(smem_u32(&bars[last_stage]), last_parity, stall, stall_cycles);
      if (__syncthreads_or(!ok)) failed = true;
    }
    tc_fence_after();
    if (!failed && warp < 4 && in_window > 0) {
      float v[32];
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      tc_load32(lane_base, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] += (double)v[i];
      tc_load32(lane_base + kLoRow, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] += (double)v[i];
    }
    in_window = 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };

  // prologue: nraw - 1 chunks in flight
  for (int p = 0; p < nraw - 1; ++p) issue(blockIdx.x + (long long)p * gridDim.x, p);

  for (long long ch = blockIdx.x; ch < nchunks && !failed; ch += gridDim.x) {
    const int stage = it & 1;
    const uint32_t use = (uint32_t)(it >> 1);
    unsigned char* st = stage_base + stage * kStage;
    const int slot = it % nraw;
    issue(ch + (long long)(nraw - 1) * gridDim.x, (it + nraw - 1) % nraw);
    // this thread's copies of chunk ch have landed (newer groups may still fly)
    if (nraw == 4) cp_async_wait<3>();
    else if (nraw == 3) cp_async_wait<2>();
    else if (nraw == 2) cp_async_wait<1>();
    else cp_async_wait<0>();
    bool ok = true;
    if (use >= 1) ok = mbar_wait(smem_u32(&bars[stage]), (use - 1) & 1, stall, stall_cycles);  // stage free again
    if (__syncthreads_or(!ok)) {  // also makes every thread's raw copies visible
      failed = true;
      break;
    }
    // split raw rows into TF32 hi / lo parts; consecutive threads take
    // consecutive rows (conflict-free 16-byte reads and writes)
    const unsigned char* raw = raw_base + (uint32_t)slot * raw_stage_bytes;
    const long long k0 = ch * kTcK;
    for (int idx = tid; idx < rows * (kTcK / 4); idx += kTcThreads) {
      const int row = idx % rows, q = idx / rows;
      float4 x = *reinterpret_cast<const float4*>(raw + (uint32_t)row * kRawPitch + 16u * q);
      float4 hi, lo;
      if (row < ma) {
        split_tf32(x.x, hi.x, lo.x);
        split_tf32(x.y, hi.y, lo.y);
        split_tf32(x.z, hi.z, lo.z);
        split_tf32(x.w, hi.w, lo.w);
        *reinterpret_cast<float4*>(st + tile_off(row, 4 * q)) = hi;
        if (packed) *reinterpret_cast<float4*>(st + tile_off(kPackRows + row, 4 * q)) = lo;
        else *reinterpret_cast<float4*>(st + kTileA + tile_off(row, 4 * q)) = lo;
      } else {
        const int j = row - ma;
        if (g5b && k0 + 4 * q >= half_k) x = make_float4(-x.x, -x.y, -x.z, -x.w);
        const float4 xt = make_float4(x.y, -x.x, x.w, -x.z);
        float4 thi, tlo;
        split_tf32(x.x, hi.x, lo.x);
        split_tf32(x.y, hi.y, lo.y);
        split_tf32(x.z, hi.z, lo.z);
        split_tf32(x.w, hi.w, lo.w);
        split_tf32(xt.x, thi.x, tlo.x);
        split_tf32(xt.y, thi.y, tlo.y);
        split_tf32(xt.z, thi.z, tlo.z);
        split_tf32(xt.w, thi.w, tlo.w);
        unsigned char* bt = st + offB;
        *reinterpret_cast<float4*>(bt + tile_off(j, 4 * q)) = hi;
        *reinterpret_cast<float4*>(bt + tile_off(mb + j, 4 * q)) = thi;
        *reinterpret_cast<float4*>(bt + tile_off(kLoRow + j, 4 * q)) = lo;
        *reinterpret_cast<float4*>(bt + tile_off(kLoRow + mb + j, 4 * q)) = tlo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      // the descriptor's address field is addr >> 4 in its low bits (all of
      // this CTA's shared memory stays below 2^18 bytes), so tiles and K
      // steps are plain offsets of one base descriptor
      const uint64_t d_a0 = smem_desc(smem_u32(st));
      const uint64_t d_a1 = d_a0 + (kTileA >> 4), d_b = d_a0 + (offB >> 4);
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint64_t o = (uint64_t)kk * (256 >> 4);  // 8 floats = two core matrices along K
        const uint32_t acc_in = (in_window > 0 || kk > 0) ? 1u : 0u;
        tc_mma(tmem, d_a0 + o, d_b + o, acc_in);
        if (!packed) tc_mma(tmem, d_a1 + o, d_b + o, 1u);
      }
      tc_commit(smem_u32(&bars[stage]));
    }
    last_stage = stage;
    last_parity = use & 1;
    ++it;
    ++in_window;
    if (in_window == kFlush) flush();
  }
  cp_async_wait<0>();  // no copy may still target shared memory when the CTA exits
  if (!failed) flush();
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    // bounded wait (no stall) for this CTA's own MMAs before releasing tensor memory
    if (last_stage >= 0) mbar_wait(smem_u32(&bars[last_stage]), last_parity);
  }
  if (!failed && packed) {
    // lanes 64 + i hold the lo.hi and lo.lo products of row i: add them into lane i
    // (the stages are free: the last flush waited for every MMA)
    double* fold = reinterpret_cast<double*>(stage_base);
    if (tid >= kPackRows && tid < 2 * kPackRows) {
#pragma unroll
      for (int i = 0; i < 32; ++i) fold[(tid - kPackRows) * 33 + i] = acc[i];
    }
    __syncthreads();
    if (tid < kPackRows) {
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] += fold[tid * 33 + i];
    }
  }
  if (!failed && warp < 4) {
    const int row = tid;  // warps 0-3: lane quarter = rows 0..127
    if (row < ma) {  // acc[j] = Re, acc[mb + j] = Im of C_row,j (static indices keep acc in registers)
      double* pd = reinterpret_cast<double*>(partial);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < mb) pd[2 * (((long long)row * mb + c) * gridDim.x + blockIdx.x)] = acc[c];
        else if (c < 2 * mb) pd[2 * (((long long)row * mb + c - mb) * gridDim.x + blockIdx.x) + 1] = acc[c];
      }
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
int tc_gram_max_rhs() { return kLoRow / 2; }

cudaError_t launch_tc_gram(const void* A, int ma, const void* B, int mb, int64_t V, int g5b, double2* partial,
                           int nblk, int* err, const int* stall, long long stall_cycles, cudaStream_t st) {
  if (ma < 1 || ma > kTcM || mb < 1 || 2 * mb > kLoRow) return cudaErrorInvalidValue;
  const uint32_t nraw = raw_stages(ma, ma + mb);
  const uint32_t smem = 2 * stage_bytes(ma) + kCtrl + nraw * (uint32_t)(ma + mb) * kRawPitch;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_gram<<<nblk, kTcThreads, smem, st>>>(static_cast<const float*>(A), ma, static_cast<const float*>(B), mb,
                                            24LL * V, g5b, partial, err, (int)nraw, stall, stall_cycles);
  return cudaGetLastError();
}

}  // namespace ov
