// Host-side declarations shared by the translation units of the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ov {

// Storage precision of an operator instance (links and the spinors of its
// recurrence are stored in this type; arithmetic is FP64 for OP_F64 and FP32
// otherwise).
enum OpPrec { OP_F64 = 0, OP_F32 = 1, OP_F16 = 2, OP_B16 = 3 };

inline int spinor_bytes_per_site(OpPrec p) {
  return p == OP_F64 ? 192 : p == OP_F32 ? 96 : 48;
}
// bytes of one direction's link at one site as stored
inline int link_bytes_per_site_dir(OpPrec p, int lrec = 12) {
  return p == OP_F64 ? 144 : p == OP_F32 ? 48 : (lrec == 18 ? 36 : 24);
}

struct LatticeH {
  int L[4];
  int64_t V;
  int antiperiodic_t;
};

// Fused epilogue of one stencil application:
//   r   = D_W x                      (wilson = 1)
//       = gamma5 (D_W - m_w) x = K x (wilson = 0)
//   out = c0 * y + G( s1 * r + sum_j w[j] * v[j] + wz * z ),  G = gamma5 if g5_out else 1
// Null v[j] / z / y are skipped.  The stencil input x and v[j] are in the
// operator's storage p; z, y and out are in out_prec (p itself, or FP32 for a
// 16-bit operator whose results are assembled in FP32).
struct EpiArgs {
  int wilson = 0;
  double m_w = 1.5;
  int g5_out = 0;
  double s1 = 1.0;
  const void* v[3] = {nullptr, nullptr, nullptr};
  double w[3] = {0.0, 0.0, 0.0};
  const void* z = nullptr;
  double wz = 0.0;
  const void* y = nullptr;
  double c0 = 0.0;
  int keep_half = -1;  // 0: spins 2, 3 of G5(...) set to zero (chirality +), 1: spins 0, 1; -1: none
};

// Launch shape and link layout of the stencil (chosen per operator by the
// autotuner): threads per block over an (x, y) plane, a register cap (minb
// 1 / 2 / 3 / 4 = none / 128 / 80 / 64 registers), right-hand sides per thread, and for 16-bit links 12 (rows 0, 1; row 2 rebuilt)
// or 18 stored reals.
struct DslashCfg {
  int tpb = 128;
  int minb = 2;
  int lrec = 12;
  int rt = 1;  // right-hand sides per thread (each link loaded once for all of them)
  int slab = 0;  // > 0: the slab kernel (16-bit storage, 12-real links) on this many persistent CTAs
  int async = 0;  // 16-bit storage, 12-real links, one RHS per thread: 1 = operands staged in shared memory
                  // by asynchronous copies (spinors and links), 2 = spinors only (dslash_async.cuh)
  int brick = 0;  // 1: a block covers an 8 x 4 x (tpb / 32) brick of sites (Lx % 8 = Ly % 4 = 0,
                  // Lz % (tpb / 32) = 0) instead of consecutive sites of an (x, y) plane
  int* err = nullptr;  // slab kernel: set to 1 (device-visible memory) if a bulk copy did not land in time
  const int* stall = nullptr;  // slab kernel, testing: a device flag nothing sets, waited on for stall_cycles
  long long stall_cycles = 0;  // by every pipeline wait, which then reports expiry (ov_test_wait_expiry)
};

// Whether blocks of tpb threads can be mapped onto 8 x 4 x (tpb / 32) bricks.
inline bool brick_lattice_ok(const LatticeH& g, int tpb) {
  const int bz = tpb / 32;
  return tpb % 32 == 0 && bz >= 1 && g.L[0] % 8 == 0 && g.L[1] % 4 == 0 && g.L[2] % bz == 0;
}

// Whether the slab kernel takes this lattice (Lx Ly a multiple of 32, at most 640).
bool slab_lattice_ok(const LatticeH& g);
// Resident slab CTAs per SM on this lattice (0: not available).
int slab_ctas_per_sm(const LatticeH& g);

// Optional L2 access-policy window (persisting) applied to stencil launches
// whose links pointer is `base`.
struct L2Window {
  const void* base = nullptr;
  size_t bytes = 0;
};
L2Window& l2_window();

// Returns false if the (minb, rt) variant is not compiled for this storage.
bool launch_dslash(OpPrec p, OpPrec out_prec, const DslashCfg& cfg, const LatticeH& g, const void* links,
                   const void* in, void* out, const EpiArgs& e, int nrhs, cudaStream_t st);

// ---- vector kernels (blas.cu) ---------------------------------------------
// Interface formats: complex128 / complex64 AoS [nrhs][V][4][3].
enum IfaceType { IF_C128 = 0, IF_C64 = 1 };

// internal <- interface, out = scale * (g5 ? gamma5 : 1) in
void launch_pack_spinor(OpPrec p, IfaceType it, const LatticeH& g, const void* in, void* out, int nrhs,
                        double scale, int g5, cudaStream_t st);
// interface <- internal
void launch_unpack_spinor(OpPrec p, IfaceType it, const LatticeH& g, const void* in, void* out, int nrhs,
                          double scale, cudaStream_t st);
// links complex128 [4][V][3][3] -> internal storage (lrec 12 or 18 reals for
// 16-bit storage; FP64 always 18, FP32 always 12)
void launch_pack_links(OpPrec p, int lrec, const LatticeH& g, const void* in, void* out, cudaStream_t st);
// FP64 packed links -> complex128 [4][V][3][3]
void launch_unpack_links_f64(const LatticeH& g, const void* packed, void* out, cudaStream_t st);

// Number of blocks every reduction kernel uses (fixed, so that results are
// bitwise reproducible).
constexpr int kReduceBlocks = 608;
constexpr int kReduceThreads = 256;

// Deflation, step 1: partial[i][blk] = sum over the block's sites of
// conj(phi_i) . ((g5 ? gamma5 : 1) psi), i < n_ev; complex, per-site products
// in the storage's arithmetic, sums over sites in FP64.  phi (n_ev vectors
// of V sites, back to back) and psi in storage pv (FP64 or FP32).
void launch_defl_dot(OpPrec pv, const LatticeH& g, const void* evecs, int n_ev, const void* psi,
                     int g5, double2* partial, cudaStream_t st);
// sum partial[i][0..nblk) in a fixed order -> out[i]
void launch_reduce_partials(const double2* partial, int n, int nblk, double2* out, cudaStream_t st);
// Deflation, step 2 (and conversion into the recurrence's storage):
//   psi_perp = scale * (G psi - sum_i c_i phi_i),   d = scale * sum_i sgn_i c_i phi_i
// (d skipped when null; G = gamma5 if g5).
// phi, psi and d are in storage pv (FP64 or FP32), psi_perp in pp (the
// operator's recurrence storage); c_i is read at c[i * cstride].
void launch_defl_combine(OpPrec pv, OpPrec pp, const LatticeH& g, const void* evecs, int n_ev,
                         const double2* c, int cstride, const double* sgn, const void* psi, int g5, double scale,
                         void* psi_perp, void* d, cudaStream_t st);

// Several right-hand sides with FP32 vectors (n_ev <= 128): c[i*nrhs + r] from
// the batched projection; psi_perp in pp (FP32 / FP16 / BF16), d in FP32.
void launch_defl_combine_multi(OpPrec pp, const LatticeH& g, const void* evecs, int n_ev, const double2* c, int nrhs,
                               const double* sgn, const void* psi, int g5, double scale, void* psi_perp, void* d,
                               cudaStream_t st);

// BLAS-1 on internal spinors of storage p: nrhs fields of V sites each,
// stored back to back.  Reductions leave one double2 per block in partial[]
// (complex dot: re/im; norm: .x), to be summed by launch_reduce_partials.
void launch_dot_partial(OpPrec p, const void* a, const void* b, int64_t V, int nrhs, double2* partial,
                        cudaStream_t st);
void launch_norm2_partial(OpPrec p, const void* a, int64_t V, int nrhs, double2* partial, cudaStream_t st);
// x += alpha p ; r -= alpha q ; partial |r|^2
void launch_cg_update_xr(OpPrec p, void* x, void* r, const void* pv, const void* q, double alpha, int64_t V,
                         int nrhs, double2* partial, cudaStream_t st);
// p = r + beta p
void launch_cg_update_p(OpPrec p, void* pv, const void* r, double beta, int64_t V, int nrhs, cudaStream_t st);
// out = a*x + b*y (out may alias x or y; y may be null => out = a*x)
void launch_axpby(OpPrec p, double a, const void* x, double b, const void* y, void* out, int64_t V, int nrhs,
                  cudaStream_t st);
// y = y + a x with complex a
void launch_caxpy(OpPrec p, double2 a, const void* x, void* y, int64_t V, int nrhs, cudaStream_t st);
// One step of the shifted-unitary minimal residual recursion (one RHS) on
// lazily normalised vectors: the stored V, T, Dh, Dth are the true v_j,
// v~_j, D_j, D~_j times the divisors of the previous step, W = U V.
//   X += cx Dh;  t = av V + zv Dh;  Dh = t - mt Dth;  Dth = at Dth - mc t;
//   V = av W - mt T;  T = at T - mcv W;
// partial[blk] = block sums of (|V|^2, |T|^2) of the new V and T.
struct SumrCoef {
  double2 cx;   // conj(phi_j(zeta)) / rho_{j-1}: the deferred term of X
  double av;    // 1 / rho_{j-1}: v_j = av V, D_j = av Dh
  double at;    // 1 / rho~_{j-1}: v~_j = at T, D~_j = at Dth
  double zv;    // zeta av
  double2 mt;   // m at
  double2 mc;   // conj(m)
  double2 mcv;  // conj(m) av
};
void launch_sumr_update(OpPrec p, void* v, void* vt, const void* w, void* dh, void* dth, void* x, const SumrCoef& c,
                        int64_t V, double2* partial, cudaStream_t st);
// out (storage po) = scale * in (storage pi)            (accumulate = 0)
// out (storage po) = out + scale * in (storage pi)      (accumulate = 1)
void launch_convert(OpPrec pi, OpPrec po, const void* in, void* out, int64_t V, int nrhs, double scale,
                    int accumulate, cudaStream_t st);

// ---- eigensolver block kernels (eigs.cu) ------------------------------------
// Block storage: m vectors of V sites back to back, storage OP_F64 or OP_F32.
void launch_random_block(OpPrec p, void* out, int m, int64_t V, uint64_t seed, cudaStream_t st);
// partial[(i*mb + j)*nblk + blk] = block blk's share of <A_i, G B_j>
// (G = gamma5 if g5b, else 1); ma, mb <= gram_max_vectors().
cudaError_t launch_gram(OpPrec p, const void* A, int ma, const void* B, int mb, int64_t V, double2* partial,
                        int nblk, cudaStream_t st, int g5b = 0);
int gram_max_vectors();
// out_j = sum_i Y_i Q[i*m_out + j]   (Q complex FP64 on the device; out must not alias Y)
void launch_rotate(OpPrec p, const void* Y, int m_in, const double2* Q, int m_out, void* out, int64_t V,
                   cudaStream_t st);

// ---- link derivative (force.cu) ------------------------------------------------
// G_mu(x) += sum_p w_p * (colour outer products of pair p), see force.cu.
constexpr int kMaxForcePairs = 34;
struct ForcePairs {
  const void* u[kMaxForcePairs];
  const void* v[kMaxForcePairs];
  double w[kMaxForcePairs];
  int n = 0;
};
// G: complex [4][9][V] in the arithmetic type of p (OP_F64 or OP_F32); pair
// vectors in the same storage.
void launch_force_pairs(OpPrec p, const LatticeH& g, const void* links, const ForcePairs& pairs, void* G,
                        cudaStream_t st);
// out: complex128 AoS [4][V][3][3] = P_TA(G^dagger)
void launch_force_finish(OpPrec p, const void* G, int64_t V, void* out, cudaStream_t st);

// ---- tensor-core deflation projection (tc_gram.cu) ----------------------------
// partial[(i*mb + j)*nblk + blk] as launch_gram, for FP32 vectors, computed
// with tcgen05 (TF32 x 3 split products); ma <= tc_gram_max_rows(),
// mb <= tc_gram_max_rhs().  *err is set to 1 if a bounded wait expired.
// stall (testing; null normally): a device flag that nothing sets, on which
// every pipeline wait first waits up to stall_cycles and then reports expiry;
// the drain before exit waits as usual.
cudaError_t launch_tc_gram(const void* A, int ma, const void* B, int mb, int64_t V, int g5b, double2* partial,
                           int nblk, int* err, const int* stall, long long stall_cycles, cudaStream_t st);
int tc_gram_max_rows();
int tc_gram_max_rhs();

}  // namespace ov
