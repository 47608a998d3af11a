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
// Pipeline per CTA (512 threads, warp-specialised): 15 worker warps copy raw
// 64-float chunks of every row into a ring of up to six shared-memory
// buffers with cp.async (sixteen lanes per row's 256 bytes; several chunks in
// flight), meet at a named barrier of the worker warps once a chunk has
// landed, and split their fixed 16-byte pieces (eight consecutive lanes on
// eight consecutive rows) into TF32 hi / lo parts in one of two or three MMA
// stages (canonical no-swizzle K-major layout, 8-row x 16-byte core
// matrices), then arrive on the stage's "filled" mbarrier.  Lane 0 of the
// last warp waits on it, issues the chunk's 8 (or 16) MMAs and commits them
// to the stage's "consumed" mbarrier, which the workers wait on before
// refilling the stage.  The whole CTA synchronises only when it moves the
// tensor-memory accumulator into FP64 registers (every 64 chunks).  Every
// mbarrier wait is bounded (about a second); on expiry a thread raises a
// shared abort flag, every thread runs the rest of its iterations without
// work (so the barriers still match), the kernel records an error flag,
// waits (bounded) for its own copies and MMAs in flight, frees its tensor
// memory and returns.
#include "common.cuh"
#include "internal.h"

namespace ov {

namespace {

constexpr int kTcM = 128;      // MMA M: A tile rows
constexpr int kTcN = 64;       // MMA N: B tile rows (hi parts in 0..31, lo parts in 32..63)
constexpr int kLoRow = 32;     // first B row of the lo parts
constexpr int kPackRows = 64;  // n_ev <= 64: a_i lo in A row 64 + i
constexpr int kTcK = 64;       // floats per chunk and stage
constexpr int kWorkerWarps = 15;         // copy and split
constexpr int kWorkers = 32 * kWorkerWarps;
constexpr int kTcThreads = kWorkers + 32;  // + one warp whose lane 0 issues the MMAs
constexpr int kRawPitch = kTcK * 4 + 16;  // bytes per raw row (padded: conflict-free 16-byte reads)
constexpr int kRawStagesMax = 6;          // chunks in flight (cp.async ring of raw FP32 rows)
constexpr int kFlush = 64;     // chunks per tensor-memory accumulation window
constexpr int kTmemCols = 64;

constexpr uint32_t kTileA = kTcM * kTcK * 4;  // bytes of one A tile
constexpr uint32_t kTileB = kTcN * kTcK * 4;
constexpr uint32_t kCtrl = 1024;                     // mbarriers, tensor-memory address
__host__ __device__ inline uint32_t stage_bytes(int ma) { return (ma <= kPackRows ? 1u : 2u) * kTileA + kTileB; }
// dynamic shared memory: nstage MMA stages, control block, raw ring of
// nraw chunks.  Three MMA stages when they leave room for a ring of at least
// four chunks (the hi / lo-packed tile), else two.
constexpr uint32_t kSmemMax = 227u * 1024u;
inline uint32_t raw_stages(int ma, int rows, int nstage) {
  const uint32_t avail = kSmemMax - (uint32_t)nstage * stage_bytes(ma) - kCtrl;
  const uint32_t per = (uint32_t)rows * kRawPitch;
  const uint32_t n = avail / per;
  return n < 1 ? 1 : (n > (uint32_t)kRawStagesMax ? (uint32_t)kRawStagesMax : n);
}
inline int mma_stages(int ma, int rows) {
  const uint64_t need3 = 3ull * stage_bytes(ma) + kCtrl + 4ull * (uint64_t)rows * kRawPitch;
  return need3 <= kSmemMax ? 3 : 2;
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

// One try_wait with a suspend-time hint: a thread whose phase is not yet
// complete is parked (up to ~0.1 ms) instead of spinning, so the warps that
// wait do not take issue slots from the ones that work.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within ~2^31 cycles or
// another thread of the CTA raised *abort.  stall (testing, see
// ov_test_wait_expiry): a device flag that nothing sets; when given, the wait
// first waits up to stall_cycles for it, runs out and reports failure as an
// expired wait would.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort,
                                          const volatile int* stall = nullptr, long long stall_cycles = 0) {
  const long long t0 = clock64();
  if (stall != nullptr) {
    while (*stall == 0) {
      if (clock64() - t0 > stall_cycles) return false;
    }
  }
  while (!mbar_test(bar, parity)) {
    if ((abort != nullptr && *abort != 0) || clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// 16 warps of <= 128 registers: each scheduler's quarter of the register file holds its four warps
template <int NI>  // 16-byte pieces per worker thread and chunk
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gram(const float* __restrict__ A, int ma, const float* __restrict__ B, int mb, long long K, int g5b,
              double2* __restrict__ partial, int* __restrict__ err, int nstage, int nraw, const int* stall,
              long long stall_cycles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const bool packed = ma <= kPackRows;
  const uint32_t kStage = stage_bytes(ma);
  const uint32_t offB = kStage - kTileB;  // B tile after the one or two A tiles
  unsigned char* stage_base = smem;
  // bars[s]: the MMAs reading stage s completed (tcgen05.commit); bars[4 + s]:
  // stage s filled (one arrival per worker warp); s < nstage <= 3
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + nstage * kStage);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + nstage * kStage + 64);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + nstage * kStage + 128);
  unsigned char* raw_base = smem + nstage * kStage + kCtrl;
  const int rows = ma + mb;
  const int nitem = ((rows + 7) / 8) * 128;  // item space: 8-row groups x 16 pieces
  const uint32_t raw_stage_bytes = (uint32_t)rows * kRawPitch;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp < kWorkerWarps;
  const bool issuer = warp == kWorkerWarps && lane == 0;
  const long long half_k = K / 2;  // gamma5 flips the second half of each vector (spins 2, 3)

  // zero the MMA stages once: rows no chunk writes stay zero
  for (uint32_t i = tid; i < (uint32_t)nstage * kStage / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(stage_base)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int b = 0; b < nstage; ++b) {
      mbar_init(smem_u32(&bars[b]), 1);
      mbar_init(smem_u32(&bars[4 + b]), kWorkerWarps);
    }
    *abort_flag = 0;
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

  const long long nchunks = (K + kTcK - 1) / kTcK;  // K <= 24 * 2^27: nchunks < 2^26
  // chunks of this CTA: blockIdx.x + it * gridDim.x for it < niter (the same for every thread)
  const int niter = blockIdx.x < nchunks ? (int)((nchunks - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  bool failed = false;
  const long long kstep = (long long)gridDim.x * kTcK;  // k0 advance per iteration

  // A worker's pieces are fixed, one set for copying and one for splitting,
  // each worked out once (everything but the chunk offset k0 is fixed):
  //  - copy item c = tid + kWorkers m is piece c % 16 of row c / 16: sixteen
  //    lanes cover one row's 256 contiguous bytes, so each warp copies whole
  //    lines of two rows (fewer, fuller memory requests);
  //  - split item i = tid + kWorkers m is piece (i % 128) / 8 of row
  //    (i / 128) * 8 + i % 8: eight consecutive lanes take eight consecutive
  //    rows of one piece (conflict-free tile stores).
  // The two differ, so a named barrier of the worker warps separates the
  // copies of a chunk from its split.
  const char* csrc[NI];
  uint32_t craw[NI];
  long long clim[NI];
  bool cval[NI];
  uint32_t iraw[NI], io0[NI], io1[NI], io2[NI], io3[NI];
  long long iglim[NI];
  int ikind[NI];  // 0: none, 1: eigenvector row (A), 2: right-hand-side row (B)
#pragma unroll
  for (int m = 0; m < NI; ++m) {
    const int c = tid + kWorkers * m;
    const int crow = c >> 4, cq = c & 15;
    cval[m] = worker && crow < rows;
    csrc[m] = reinterpret_cast<const char*>(crow < ma ? A + (long long)crow * K : B + (long long)(crow - ma) * K) +
              16 * cq;
    craw[m] = (uint32_t)crow * kRawPitch + 16u * cq;
    clim[m] = K - 4 * cq;  // piece cq of the chunk at k0 lies inside K when k0 < K - 4 cq
    const int i = tid + kWorkers * m;
    const int row = (i >> 7) * 8 + (i & 7), q = (i & 127) >> 3;
    ikind[m] = (!worker || i >= nitem || row >= rows) ? 0 : (row < ma ? 1 : 2);
    const int jb = row - ma;
    iraw[m] = (uint32_t)row * kRawPitch + 16u * q;
    iglim[m] = half_k - 4 * q;  // piece q lies in the gamma5-flipped half when k0 >= half_k - 4 q
    if (ikind[m] == 1) {
      io0[m] = tile_off(row, 4 * q);
      io1[m] = packed ? tile_off(kPackRows + row, 4 * q) : kTileA + tile_off(row, 4 * q);
      io2[m] = io3[m] = 0;
    } else {
      io0[m] = offB + tile_off(jb, 4 * q);
      io1[m] = offB + tile_off(mb + jb, 4 * q);
      io2[m] = offB + tile_off(kLoRow + jb, 4 * q);
      io3[m] = offB + tile_off(kLoRow + mb + jb, 4 * q);
    }
  }

  // (ring slots and k0 are passed in: they advance by counters, never by a division)
  auto issue = [&](bool valid, long long k0, int slot) {  // chunk at k0 into raw slot `slot`
    if (!failed && valid) {
      const uint32_t dst0 = smem_u32(raw_base + (uint32_t)slot * raw_stage_bytes);
#pragma unroll
      for (int m = 0; m < NI; ++m) {
        if (!cval[m]) continue;
        const bool ok = k0 < clim[m];  // zero-filled past K
        cp_async16(dst0 + craw[m], ok ? csrc[m] + 4 * k0 : reinterpret_cast<const char*>(A), ok ? 16u : 0u);
      }
    }
    cp_async_commit();
  };
  // this thread's copies of chunk it have landed (groups committed: chunks up to it + nraw - 2)
  auto raw_wait = [&]() {
    switch (nraw) {
      case 6: cp_async_wait<4>(); break;
      case 5: cp_async_wait<3>(); break;
      case 4: cp_async_wait<2>(); break;
      case 3: cp_async_wait<1>(); break;
      default: cp_async_wait<0>(); break;
    }
  };
  auto worker_sync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory"); };
  // split this worker's pieces of the chunk at k0 (raw slot `slot`) into TF32 hi / lo parts in stage st
  auto split = [&](long long k0, int slot, unsigned char* st) {
    const unsigned char* raw = raw_base + (uint32_t)slot * raw_stage_bytes;
#pragma unroll
    for (int m = 0; m < NI; ++m) {
      if (ikind[m] == 0) continue;
      float4 x = *reinterpret_cast<const float4*>(raw + iraw[m]);
      float4 hi, lo;
      if (ikind[m] == 1) {
        split_tf32(x.x, hi.x, lo.x);
        split_tf32(x.y, hi.y, lo.y);
        split_tf32(x.z, hi.z, lo.z);
        split_tf32(x.w, hi.w, lo.w);
        *reinterpret_cast<float4*>(st + io0[m]) = hi;
        *reinterpret_cast<float4*>(st + io1[m]) = lo;
      } else {
        if (g5b && k0 >= iglim[m]) x = make_float4(-x.x, -x.y, -x.z, -x.w);
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
        *reinterpret_cast<float4*>(st + io0[m]) = hi;
        *reinterpret_cast<float4*>(st + io1[m]) = thi;
        *reinterpret_cast<float4*>(st + io2[m]) = lo;
        *reinterpret_cast<float4*>(st + io3[m]) = tlo;
      }
    }
  };

  // FP64 sums of the hi-column (0..31) and lo-column (32..63) accumulators of this thread's lane
  double acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.0;
  int in_window = 0;  // (issuer) chunks in the current accumulation window
  int last_stage = -1;
  uint32_t last_parity = 0;
  auto raise = [&]() {
    failed = true;
    *abort_flag = 1;
  };

  long long k0_use = (long long)blockIdx.x * kTcK;  // k0 of chunk it
  if (worker)  // prologue: nraw - 1 chunks in flight
    for (int p = 0; p < nraw - 1; ++p) issue(p < niter, k0_use + p * kstep, p);
  long long k0_fill = k0_use + (long long)(nraw - 1) * kstep;  // k0 of chunk it + nraw - 1
  int stage = 0;        // it % nstage
  uint32_t use = 0;     // it / nstage
  int slot = 0;         // it % nraw: raw slot of chunk it
  int fill = nraw - 1;  // (it + nraw - 1) % nraw: raw slot of the chunk issued in iteration it
  for (int it = 0; it < niter; ++it) {
    unsigned char* st = stage_base + stage * kStage;
    if (*abort_flag) failed = true;  // another thread's wait expired: skip the rest
    if (worker) {
      if (nraw >= 2) {
        raw_wait();
        worker_sync();  // every worker's copies of chunk it landed; chunk it - 1 is split (its slot is free)
        issue(it + nraw - 1 < niter, k0_fill, fill);
      } else {  // one raw slot: copy and split in turn
        worker_sync();
        issue(true, k0_use, 0);
        cp_async_wait<0>();
        worker_sync();
      }
      if (!failed && use >= 1 &&
          !mbar_wait(smem_u32(&bars[stage]), (use - 1) & 1, abort_flag, stall, stall_cycles))  // stage free
        raise();
      if (!failed) {
        split(k0_use, slot, st);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
      }
      __syncwarp();
      if (!failed && lane == 0) mbar_arrive(smem_u32(&bars[4 + stage]));
    } else if (issuer) {
      if (!failed && !mbar_wait(smem_u32(&bars[4 + stage]), use & 1, abort_flag, stall, stall_cycles)) raise();
      if (!failed) {
        tc_fence_after();
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
        last_stage = stage;
        last_parity = use & 1;
      }
      ++in_window;
    }
    if ((it + 1) % kFlush == 0 || it + 1 == niter) {
      // window complete: its last commit covers every MMA issued so far
      if (issuer && !failed && last_stage >= 0 &&
          !mbar_wait(smem_u32(&bars[last_stage]), last_parity, abort_flag, stall, stall_cycles))
        raise();
      __syncthreads();
      if (*abort_flag) failed = true;  // uniform: no thread writes the flag between the two barriers
      tc_fence_after();
      if (!failed && warp < 4) {
        float v[32];
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        tc_load32(lane_base, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] += (double)v[i];
        tc_load32(lane_base + kLoRow, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] += (double)v[i];
      }
      tc_fence_before();
      __syncthreads();
      in_window = 0;
    }
    if (++stage == nstage) {
      stage = 0;
      ++use;
    }
    if (++slot == nraw) slot = 0;
    if (++fill == nraw) fill = 0;
    k0_use += kstep;
    k0_fill += kstep;
  }
  if (worker) cp_async_wait<0>();  // no copy may still target shared memory when the CTA exits
  const bool any_failed = __syncthreads_or(failed || *abort_flag != 0);
  if (any_failed) {
    if (tid == 0) atomicExch(err, 1);
    // bounded wait (no stall, no abort) for this CTA's own MMAs before releasing tensor memory
    if (issuer && last_stage >= 0) mbar_wait(smem_u32(&bars[last_stage]), last_parity, nullptr);
  }
  if (!any_failed && packed) {
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
  if (!any_failed && warp < 4) {
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
  const int nstage = mma_stages(ma, ma + mb);
  const uint32_t nraw = raw_stages(ma, ma + mb, nstage);
  const uint32_t smem = (uint32_t)nstage * stage_bytes(ma) + kCtrl + nraw * (uint32_t)(ma + mb) * kRawPitch;
  const int nitem = ((ma + mb + 7) / 8) * 128;
  const int ni = (nitem + kWorkers - 1) / kWorkers;  // <= 5 for 144 rows
  auto run = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<nblk, kTcThreads, smem, st>>>(static_cast<const float*>(A), ma, static_cast<const float*>(B), mb,
                                         24LL * V, g5b, partial, err, nstage, (int)nraw, stall, stall_cycles);
    return cudaGetLastError();
  };
  if (ni <= 2) return run(k_tc_gram<2>);
  if (ni <= 3) return run(k_tc_gram<3>);
  return run(k_tc_gram<5>);
}

}  // namespace ov
