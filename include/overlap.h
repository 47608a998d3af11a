/*
 * overlap.h -- C ABI of the GB300 (sm_103a) overlap Dirac operator library.
 *
 * Operator (Cundy & Lee, "Overlap fermions on GPUs", arXiv:1510.06897):
 *
 *   D[mu]   = 1/2 (1 + mu + (1 - mu) gamma5 sign(K))                               (Eq. 1)
 *   K       = gamma5 (D_W - m_W),  m_W = 1.5                                        (Sec. 2)
 *   D_W psi = 4 psi(x) - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu^)
 *                                  + (1 + gamma_mu) U_mu(x-mu^)^dagger psi(x-mu^)] (Eq. 2)
 *   sign(K) = sum_m alpha_m T_m(K)
 *             + sum_i phi_i phi_i^dagger [sign(lambda_i) - sum_m alpha_m T_m(lambda_i)] (Eq. 3)
 *
 * Reading of Eq. 3 used by every call: the polynomial is P(K) = K f_N(K^2), with
 * f_N the order-N Chebyshev interpolant of y^{-1/2} on [lo^2, hi^2] (N + 1
 * coefficients, 2N + 1 applications of K per sign apply), and the deflation is
 * applied in projected form: sign(K) psi = P(K)(1 - Phi Phi^dagger) psi
 * + sum_i sign(lambda_i) phi_i phi_i^dagger psi (equal to Eq. 3 for exact
 * eigenvectors).  Gamma basis: chiral (DeGrand-Rossi), gamma5 = diag(1,1,-1,-1).
 *
 * Layouts (all interface arrays are AoS, little-endian, C order):
 *   dims     = {Lx, Ly, Lz, Lt}, each >= 2; V = Lx Ly Lz Lt; site index
 *              s = ((t*Lz + z)*Ly + y)*Lx + x.
 *   links    complex128 [4][V][3][3]: U_mu(s) on the link s -> s+mu^, mu = x,y,z,t,
 *              colour matrix row-major.  Must be SU(3) to rounding (rows 0 and 1
 *              are stored in FP32/FP16/BF16 operators, row 2 is rebuilt).
 *   spinors  complex128 (OV_C128) or complex64 (OV_C64) [nrhs][V][4][3],
 *              [spin][colour] per site; 1 <= nrhs <= 65535.
 *   evecs    complex128 [n_ev][V][4][3], orthonormal eigenvectors of K.
 *
 * Pointers: every vector / link / evec pointer may be a device pointer or a
 * host pointer (detected with cudaPointerGetAttributes; host data is staged
 * through a context-owned device buffer with cudaMemcpyAsync).  Caller-owned
 * memory is never retained after a call returns.  All work is issued on the
 * stream given to ov_create; calls return after the result is complete.
 *
 * Errors: every call returns an ov_status; ov_last_error() gives a one-line
 * description of the last failure on that context.  Invalid arguments are
 * rejected before any device work.  A CUDA failure returns OV_ERR_CUDA.  No
 * kernel in the library waits on another block or on the host, so no call can
 * hang the device.
 *
 * Precisions (ov_create):
 *   OV_FP64        links (18 reals) and vectors FP64, FP64 arithmetic.
 *   OV_FP32        links reconstruct-12 and vectors FP32, FP32 arithmetic,
 *                  FP64 global sums.
 *   OV_MIXED_FP16  links reconstruct-12 and recurrence vectors FP16, FP32
 *                  arithmetic; deflation, assembly and solver inner vectors FP32.
 *   OV_MIXED_BF16  as OV_MIXED_FP16 with BF16 storage.
 * ov_wilson / ov_kernel / ov_sign* / ov_overlap run in the context's precision.
 * ov_solve always converges the residual of the FP64 operator (the context
 * keeps an FP64 copy of links and eigenvectors): OV_FP64 runs plain FP64 CG;
 * the other precisions run inner CG in their own precision inside an FP64
 * defect-correction loop.
 */
#ifndef OVERLAP_GB300_H
#define OVERLAP_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ov_ctx ov_ctx;

typedef enum {
  OV_OK = 0,
  OV_ERR_INVALID = 1,       /* bad argument (dims, sizes, null pointer, order, interval) */
  OV_ERR_NOMEM = 2,         /* device allocation failed */
  OV_ERR_CUDA = 3,          /* a CUDA call or kernel launch failed */
  OV_ERR_NOT_CONVERGED = 4, /* solver hit maxit; best x and its residual are still returned */
  OV_ERR_STATE = 5,         /* call needs ov_sign_config first */
  OV_ERR_NONFINITE = 6      /* (output checks on) an output vector holds NaN or Inf */
} ov_status;

typedef enum { OV_FP64 = 0, OV_FP32 = 1, OV_MIXED_FP16 = 2, OV_MIXED_BF16 = 3 } ov_prec;
typedef enum { OV_C128 = 0, OV_C64 = 1 } ov_dtype;

/* Per-context counters, reset by ov_reset_stats. */
typedef struct {
  long long kernel_launches;   /* all kernels launched by this context */
  long long dslash_launches;   /* stencil kernels (one K or D_W application each, all RHS) */
  long long sign_applies;      /* sign(K) applications (per RHS) */
  long long inner_iterations;  /* CG (SUMR) iterations in the context's precision (last solve);
                                  filter + Rayleigh-Ritz steps of the last ov_eigs */
  long long outer_iterations;  /* FP64 defect-correction steps (last ov_solve) */
  long long dslash_timed;      /* stencil launches timed while profiling was on */
  double dslash_ms;            /* their summed device time (CUDA events on the context stream) */
  int stencil_tpb;             /* autotuned stencil launch of the context-precision operator: */
  int stencil_minb;            /*   threads per block, register cap (2/3/4 = 128/80/64 regs; 5 = 72 regs,
                                      blocks of <= 64 threads), */
  int stencil_lrec;            /*   stored reals per link (12: row 2 rebuilt, 18: all) */
  int tc_gemm_launches;        /* deflation projections run on the tensor cores (several RHS, FP32 vectors) */
  int stencil_slab;            /* > 0: the tuned stencil is the slab kernel on this many persistent CTAs
                                  (stencil_tpb = Lx*Ly + 32 threads each); 0: the gather kernel */
  long long gcr_iterations;    /* GCR steps of the last ov_solve_gmresr (inner_iterations: its SUMR
                                  iterations) */
  int gmresr_order;            /* Chebyshev order of the relaxed sign in that solve */
  int stencil_async;           /* 1 / 2: the tuned stencil stages each direction's neighbour spinors and
                                  links (1) or spinors only (2) in shared memory with asynchronous
                                  copies, double-buffered; 0: loads straight into registers */
  int stencil_brick;           /* 1: its blocks cover 8 x 4 x (stencil_tpb / 32) bricks of sites;
                                  0: consecutive sites of one (x, y) plane */
  int grad_kept_terms;         /* vectors of the recurrence the last ov_sign_poly_grad kept on the device:
                                  2N + 1 (every b_k and K b_{k+1}, nothing recomputed) or its
                                  checkpoints (b_k for k = 1, 2 mod 16) */
} ov_stats;

/* Creates a context for one lattice and gauge field (Eq. 2 links).  Copies and
 * compresses the links into context-owned device memory (FP64 copy always;
 * plus the copy in `prec`).  m_w: Wilson mass of the kernel (1.5 in Sec. 2).
 * antiperiodic_t != 0: fermion boundary condition antiperiodic in t (periodic
 * otherwise).  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: OV_ERR_INVALID (null ctx/dims/links, any L < 2, V > 2^27,
 * Lz * Lt > 65535, bad prec),
 * OV_ERR_NOMEM, OV_ERR_CUDA.
 * The stencil's launch shape and (16-bit) link layout are autotuned here by
 * timing a few launches of each variant on this lattice; the environment
 * variable OV_STENCIL="tpb,minb,lrec[,rt[,async[,brick]]]" pins one gather variant, OV_STENCIL="slab"
 * the slab kernel where it applies (see ov_stats).
 * For 16-bit precisions the links are marked persisting in L2 for the stencil
 * launches (a per-process limit set here and released by ov_destroy;
 * OV_L2PIN=0 disables it). */
ov_status ov_create(ov_ctx** ctx, const int dims[4], const void* links, ov_prec prec, double m_w,
                    int antiperiodic_t, void* cuda_stream);

/* Frees all context-owned device memory.  NULL is accepted. */
ov_status ov_destroy(ov_ctx* ctx);

/* out = D_W in (Eq. 2), nrhs right-hand sides.  in and out must not overlap. */
ov_status ov_wilson(ov_ctx* ctx, const void* in, void* out, int nrhs, ov_dtype dtype);

/* out = K in = gamma5 (D_W - m_W) in (Sec. 2). */
ov_status ov_kernel(ov_ctx* ctx, const void* in, void* out, int nrhs, ov_dtype dtype);

/* Configures sign(K) (Eq. 3): Chebyshev order N >= 1 of f_N on [lo^2, hi^2]
 * with 0 < lo < hi (lo = |lambda_{n_ev+1}|, hi >= lambda_max of K), and n_ev >= 0
 * deflated eigenpairs (evals: host array of n_ev doubles; evecs: complex128
 * [n_ev][V][4][3], may be NULL when n_ev = 0).  The coefficients are computed
 * on the host in FP64; eigenvectors are copied into context-owned memory in
 * FP64 and in the context's vector precision.  sign(0) is taken as +1.
 * Errors: OV_ERR_INVALID, OV_ERR_NOMEM, OV_ERR_CUDA. */
ov_status ov_sign_config(ov_ctx* ctx, int order, double lo, double hi, const double* evals, const void* evecs,
                         int n_ev);

/* out = sign(K) in with the configuration of the last ov_sign_config.
 * OV_ERR_STATE if none. */
ov_status ov_sign_apply(ov_ctx* ctx, const void* in, void* out, int nrhs, ov_dtype dtype);

/* ov_sign_config followed by ov_sign_apply. */
ov_status ov_sign(ov_ctx* ctx, int order, double lo, double hi, const double* evals, const void* evecs, int n_ev,
                  const void* in, void* out, int nrhs, ov_dtype dtype);

/* out = D[mu] in (Eq. 1), or D[mu]^dagger in = 1/2 ((1+mu) in + (1-mu) sign(K) gamma5 in)
 * when dagger != 0.  Uses the last sign configuration (OV_ERR_STATE if none). */
ov_status ov_overlap(ov_ctx* ctx, double mu, int dagger, const void* in, void* out, int nrhs, ov_dtype dtype);

/* Solves D[mu]^dagger D[mu] x = D[mu]^dagger b by CG (one solve per RHS, all RHS
 * advanced together) until ||D^dagger b - D^dagger D x|| / ||D^dagger b|| <= tol
 * for every RHS, the residual recomputed with the FP64 operator.  x need not be
 * initialised.  iters (may be NULL): total CG iterations (inner iterations for
 * mixed precisions).  true_rel_resid (may be NULL): the largest final relative
 * residual over the RHS.  OV_ERR_NOT_CONVERGED when maxit iterations did not
 * reach tol (x holds the last iterate).  OV_ERR_STATE without a sign
 * configuration. */
ov_status ov_solve(ov_ctx* ctx, double mu, double tol, int maxit, const void* b, void* x, int nrhs,
                   ov_dtype dtype, int* iters, double* true_rel_resid);

/* Chiral-sector solve (no separate counterpart in the paper: it follows from
 * Eq. 1 and gamma5 = diag(1, 1, -1, -1)).  For a vector of one chirality,
 * P psi = psi with P = (1 + chirality gamma5)/2,
 *   D^dagger D psi = 1/4 [(1+mu)^2 + (1-mu)^2 S^2] psi + chirality/2 (1-mu^2) P S psi,
 * S = sign(K); taking S^2 = 1 gives the sector operator
 *   A = 1/4 [(1+mu)^2 + (1-mu)^2] P + chirality/2 (1-mu^2) P S P,
 * which needs ONE sign(K) application per CG iteration instead of two.  With
 * the polynomial S of Eq. 3, A differs from P D^dagger D P by the Chebyshev
 * error (S^2 = 1 only to that accuracy).  Solves A x = P b (b is projected;
 * x is returned with zero opposite-chirality components) until
 * ||P b - A x|| / ||P b|| <= tol, recomputed with the FP64 operator; the same
 * defect correction, iters and true_rel_resid as ov_solve.  D[mu]^{-1} P b is
 * then D[mu]^dagger x.  chirality: +1 or -1; |mu| < 1.  Errors: OV_ERR_INVALID
 * (bad chirality, |mu| >= 1, as ov_solve), OV_ERR_NOT_CONVERGED, OV_ERR_STATE. */
ov_status ov_solve_chiral(ov_ctx* ctx, double mu, int chirality, double tol, int maxit, const void* b, void* x,
                          int nrhs, ov_dtype dtype, int* iters, double* true_rel_resid);

/* Inner-solver controls for the mixed-precision defect correction: relative
 * tolerance of each inner solve (default 1e-5) and the maximum number of FP64
 * outer steps (default 30).  They apply to ov_solve, ov_solve_chiral and
 * ov_solve_gmresr. */
ov_status ov_set_solver_params(ov_ctx* ctx, double inner_tol, int max_outer);

/* Shifted-unitary minimal residual solve of D[mu] x = b (the SUMR named in
 * Sec. 2 as the inner solver of GMRESR(eigSUMR)).  Eq. 1 reads
 * D[mu] = (1-mu)/2 (U - zeta) with U = gamma5 sign(K) and
 * zeta = -(1+mu)/(1-mu); the iterate after k products with U is the minimal
 * residual one over the Krylov space of U when U is unitary, built by the
 * Szego recursion of U's orthonormal polynomials (short recurrences, six
 * vectors, one sign(K) application per iteration; the new Krylov pair is
 * normalised by its computed norms, which keeps the recursion stable for the
 * polynomial sign).  Runs in the context's precision with the configured
 * sign (no defect correction) until the estimate 1/sqrt(s_k) of
 * ||b - D x|| / ||b|| is <= tol for every RHS, or maxit iterations (tol = 0:
 * exactly maxit).  iters (may be NULL): iterations; est_rel_resid (may be
 * NULL): the largest final estimate (exact for unitary U; with the
 * polynomial sign it tracks the true residual).  Errors: OV_ERR_INVALID
 * (|mu| >= 1, tol < 0, maxit < 0, as ov_solve), OV_ERR_STATE,
 * OV_ERR_NOT_CONVERGED if the recursion produced a non-finite value. */
ov_status ov_sumr(ov_ctx* ctx, double mu, double tol, int maxit, const void* b, void* x, int nrhs, ov_dtype dtype,
                  int* iters, double* est_rel_resid);

/* GMRESR for D[mu] x = b (Sec. 2: recursive GMRES preconditioned by a
 * low-accuracy SUMR solve with a relaxed sign function).  Three levels:
 * FP64 defect correction on D[mu] (as ov_solve, on D itself); inside it GCR
 * on D[mu] with the configured sign -- in FP32 for OV_MIXED_FP16 /
 * OV_MIXED_BF16 contexts (an FP32 copy of the operator is built from the
 * context's FP64 links on the first call and kept; see
 * ov_set_gmresr_fp32_level), in the context precision otherwise -- its
 * directions kept and orthogonalised (up to max_dirs, then restarted); each
 * direction an ov_sumr-type solve with a LOWER-order Chebyshev polynomial on
 * the same interval (the relaxed sign; see ov_set_gmresr_params).  Stops when
 * ||b - D x|| / ||b|| <= tol for every RHS, recomputed with the FP64
 * operator.  iters (may be NULL): total SUMR iterations; ov_stats counts the
 * GCR steps (gcr_iterations) and FP64 passes (outer_iterations).
 * true_rel_resid, errors: as ov_solve; OV_ERR_INVALID for |mu| >= 1. */
ov_status ov_solve_gmresr(ov_ctx* ctx, double mu, double tol, int maxit, const void* b, void* x, int nrhs,
                          ov_dtype dtype, int* iters, double* true_rel_resid);

/* An FP32 copy of the operator beside the 16-bit one of an OV_MIXED_FP16 /
 * OV_MIXED_BF16 context, for ov_solve_gmresr: its GCR level then runs with
 * this FP32 operator (configured order) while the inner SUMR solves stay on
 * the 16-bit one, so each FP64 defect-correction pass gains about the FP32
 * accuracy instead of the 16-bit one and fewer FP64 passes are needed.
 * ov_solve_gmresr builds this copy by itself on its first call (from the
 * context's FP64 links); calling this first only moves that cost here.
 * links: the field given to ov_create, same layout (host or device).  The
 * deflation eigenvectors come from the last ov_sign_config (converted from
 * its FP64 copy) or the next one.  Costs FP32 links, eigenvectors and work
 * vectors and one stencil autotuning.  No effect on OV_FP64 / OV_FP32
 * contexts and on a second call (OV_OK).  Errors: OV_ERR_INVALID (null
 * ctx or links), OV_ERR_NOMEM, OV_ERR_CUDA (the context keeps working without
 * the FP32 copy). */
ov_status ov_enable_fp32_operator(ov_ctx* ctx, const void* links);

/* Whether ov_solve_gmresr on an OV_MIXED_FP16 / OV_MIXED_BF16 context runs
 * its GCR level on the FP32 copy of the operator (on != 0, the default) or
 * in the storage precision (0; an FP32 copy already made is freed).  Measured
 * at 24^3 x 48, FP16, mu = 0.02: 2 FP64 passes instead of 4 and 3.1 s
 * instead of 4.3 s.  No effect on other precisions.  Errors: OV_ERR_INVALID
 * (null ctx), OV_ERR_CUDA. */
ov_status ov_set_gmresr_fp32_level(ov_ctx* ctx, int on);

/* GMRESR controls.  inner_order: Chebyshev order of the relaxed sign of the
 * inner SUMR solves (0, the default: the smallest order whose sign error
 * max |sqrt(y) f_N(y) - 1| on [lo^2, hi^2] is <= 1e-2; never above the
 * configured order).  inner_tol: estimate at which an inner solve stops
 * (default 0.1).  inner_maxit: iterations per inner solve (default 1000).
 * max_dirs: GCR directions kept before a restart (1..64, default 12; each
 * costs two vectors per RHS in the context's vector precision).
 * OV_ERR_INVALID otherwise. */
ov_status ov_set_gmresr_params(ov_ctx* ctx, int inner_order, double inner_tol, int inner_maxit, int max_dirs);

/* Computes the n_ev eigenpairs of K of smallest |lambda| (the input of the
 * deflation in Eq. 3; Sec. 2 uses a polynomial-preconditioned Lanczos), by
 * Chebyshev-filtered block subspace iteration on K^2 followed by Rayleigh-Ritz
 * with K, in FP64 arithmetic for all inner products.  evals: host, n_ev
 * doubles, ascending |lambda|; evecs: complex128 [n_ev][V][4][3] (host or
 * device).  tol: relative eigen-residual ||K phi - lambda phi|| <= tol * lambda_max.
 * lambda_max_out (may be NULL): an upper bound of |lambda| of K.  max_iter
 * counts filter + Rayleigh-Ritz steps (filter degree 96 on K^2; the
 * environment variable OV_EIGS_DEGREE overrides it, 4 .. 256) on a block of
 * max(n_ev + 8, 2.5 n_ev) vectors, at most 128 (so n_ev <= 120).
 * Errors: OV_ERR_INVALID, OV_ERR_NOT_CONVERGED (best pairs returned; also when
 * the filtered block stops being finite, with no pairs written). */
ov_status ov_eigs(ov_ctx* ctx, int n_ev, double tol, int max_iter, double* evals, void* evecs,
                  double* lambda_max_out);

/* The quadratic form S = chi^dagger P(K) chi, P(K) = K f_N(K^2) the
 * undeflated polynomial of Eq. 3 on [lo^2, hi^2] (the same order and interval
 * as ov_sign_poly_grad; the context's sign configuration is neither needed nor
 * changed).  chi: one spinor in `dtype` (host or device).  *s_out (host)
 * receives S (real: P(K) is Hermitian), summed in FP64.  p_chi (may be NULL):
 * receives P(K) chi in `dtype`, whose double is the derivative of S with
 * respect to chi.  Runs the Clenshaw recurrence of Eq. 3 (2N + 2 stencil
 * launches) and one FP64 inner product.  Errors: OV_ERR_INVALID (null chi or
 * s_out, order < 1, not 0 < lo < hi, a context that is neither OV_FP64 nor
 * OV_FP32), OV_ERR_NOMEM, OV_ERR_CUDA. */
ov_status ov_sign_poly_quad(ov_ctx* ctx, int order, double lo, double hi, const void* chi, void* p_chi,
                            ov_dtype dtype, double* s_out);

/* Gradient of S = chi^dagger P(K) chi, P(K) = K f_N(K^2) the undeflated
 * polynomial of Eq. 3 on [lo^2, hi^2], with respect to every link:
 * grad_links complex128 [4][V][3][3] receives F_mu(x) in su(3) with
 * dS/deps = sum Re tr(X^dagger F) for U -> exp(eps X) U.  chi: one spinor in
 * `dtype`.  Runs the Clenshaw recurrence forward, then the adjoint recurrence
 * backward.  When the 2N + 1 vectors b_k and K b_{k+1} of the forward sweep
 * fit in the allowance of ov_set_grad_memory they all stay on the device
 * (4N + 3 stencil launches); otherwise only b_k for k = 1, 2 mod 16 are kept
 * and the backward sweep recomputes the rest (about 6N launches).
 * ov_stats.grad_kept_terms says which.  Errors: OV_ERR_INVALID, OV_ERR_NOMEM,
 * OV_ERR_CUDA. */
ov_status ov_sign_poly_grad(ov_ctx* ctx, int order, double lo, double hi, const void* chi, void* grad_links,
                            ov_dtype dtype);

/* Device memory ov_sign_poly_grad may fill with the terms of the forward
 * recurrence so that it recomputes none: bytes >= 0 sets that allowance
 * (0: always checkpoint and recompute); bytes < 0 (the default) uses half the
 * device memory free at the start of each call (counting what the context
 * already holds for it).  ov_sign_poly_quad and ov_sign_poly_grad keep their
 * device vectors in the context between calls, so that repeated calls
 * allocate nothing; this call (with any value) and ov_destroy release them.
 * Errors: OV_ERR_INVALID (null ctx), OV_ERR_CUDA. */
ov_status ov_set_grad_memory(ov_ctx* ctx, long long bytes);

/* Profiling of the stencil kernel with CUDA events on the context stream;
 * device time is added to ov_stats.dslash_ms and the number of stencil
 * launches it covers to ov_stats.dslash_timed (read back whenever a call
 * synchronises).  on = 1: an event pair around every stencil launch (exact
 * per launch, but the event records slow a sign apply by a few percent);
 * on = 2: one pair around the 2N back-to-back stencil launches of each
 * Chebyshev recurrence (their summed time including the short gaps between
 * them; other stencil launches are not timed); 0: off (default). */
ov_status ov_set_profiling(ov_ctx* ctx, int on);

/* Output checks for debugging: with on != 0 every call that returns vectors
 * (ov_wilson, ov_kernel, ov_sign_apply, ov_sign, ov_overlap, the solvers,
 * ov_sumr, ov_eigs) first sums the squares of its output in FP64 on the
 * device and fails with OV_ERR_NONFINITE, writing nothing, when that sum is
 * NaN or Inf (one extra reduction pass and a read-back per call).  Off by
 * default; OV_CHECKS=1 in the environment turns it on for every context
 * created afterwards.  Errors: OV_ERR_INVALID (null ctx). */
ov_status ov_set_checks(ov_ctx* ctx, int on);

/* Testing hook for the failure path of the kernels that wait on their own
 * asynchronous work (the tensor-core deflation projection of several
 * right-hand sides and the slab stencil), whose every wait is bounded (about
 * a second) and reported instead of hanging.  With cycles > 0, each wait of
 * their copy / MMA pipelines first waits up to `cycles` clock cycles on a
 * device flag of the context that nothing ever sets, so it runs out: the
 * kernel records its error flag, waits with its normal bound for its own
 * copies and MMAs still in flight, releases its tensor memory and returns,
 * and the call reports OV_ERR_CUDA; the context stays usable.  cycles <= 0
 * turns this off (the default).  Errors: OV_ERR_INVALID (null ctx),
 * OV_ERR_NOMEM, OV_ERR_CUDA. */
ov_status ov_test_wait_expiry(ov_ctx* ctx, long long cycles);

/* True relative residual history of the last solve (ov_solve,
 * ov_solve_chiral, ov_solve_gmresr): the largest over the RHS after each
 * FP64 defect-correction pass, recomputed with the FP64 operator.  Copies up
 * to max_len values into out (host) and sets *len (may be NULL) to the
 * number of passes.  Errors: OV_ERR_INVALID (null ctx, max_len < 0, or null
 * out with max_len > 0). */
ov_status ov_get_residual_history(const ov_ctx* ctx, double* out, int max_len, int* len);

ov_status ov_get_stats(const ov_ctx* ctx, ov_stats* out);
ov_status ov_reset_stats(ov_ctx* ctx);

/* No counterpart in the paper.  D_W in (the Wilson operator of ov_wilson, FP64
 * arithmetic, the result of ov_wilson on an OV_FP64 context; D_W itself has no
 * m_W, which enters only K) for callers that cannot allocate device
 * memory at all: code embedded in a framework whose memory pool owns the
 * whole GPU, or a latency-critical loop where a cudaMalloc may block or fail.
 * No context is needed and nothing is allocated: the packed copies of links
 * and spinors go to one file-scope device array of 32 MiB, present on every
 * GPU that loads this library until the process exits.  Requirements:
 * V * (576 + 384 * nrhs) <= 32 MiB (e.g. V <= 34952 sites for one RHS), else
 * OV_ERR_INVALID; links (complex128 [4][V][3][3]), in and out (dtype
 * [nrhs][V][4][3]) in device memory of the current device, else
 * OV_ERR_INVALID (the sizes of these buffers cannot be checked here: out and
 * in must hold nrhs * 12 * V elements of dtype).  Work is issued on
 * cuda_stream (NULL = legacy default stream) and the call returns when it is
 * complete.  All calls share the array, which keeps the last call's contents
 * (each call writes everything it reads, so nothing needs clearing): calls
 * that may overlap on the GPU race and must be serialised by the caller.  The
 * first call on a device looks up the array's address with that device
 * current and caches it.  Error text: ov_last_error(NULL). */
ov_status ov_wilson_noalloc(const int dims[4], const void* links, const void* in, void* out, int nrhs,
                            ov_dtype dtype, int antiperiodic_t, void* cuda_stream);

/* Over-improved stout smearing of a gauge field (Sec. 3 prepares its
 * ensembles with 3 steps at rho = 0.1, eps = -0.25: the stout smearing of
 * Morningstar and Peardon with the over-improved staple of Moran and
 * Leinweber).  Each step replaces every link at once (from the old field) by
 *   U' = exp(A) U,  A = 1/2 (Omega - Omega^dagger) - 1/6 tr(Omega - Omega^dagger),
 *   Omega = rho [ (5 - 2 eps)/3 (6 plaquette staples) - (1 - eps)/12
 *           (18 rectangle staples: per plane and side the 1x2 rectangle out
 *           two steps and the two 2x1 rectangles with the link first or
 *           second on the long side) ] U^dagger,
 * a staple being the path-ordered product from x to x + mu^ (eps = 1: plain
 * stout; eps = 0: tree-level Symanzik staple).  No context is needed.
 * links_in, links_out: device complex128 [4][V][3][3] (the ov_create layout),
 * may be the same buffer.  steps >= 0 (0 copies).  FP64 throughout; two
 * temporary link fields are allocated and freed inside the call.  Work runs on
 * cuda_stream (NULL = legacy default stream) and the call returns when it is
 * complete.  Errors (text: ov_last_error(NULL)): OV_ERR_INVALID (null or host
 * pointers, an extent < 2, V > 2^27, steps < 0, non-finite rho or eps),
 * OV_ERR_NOMEM, OV_ERR_CUDA. */
ov_status ov_stout_smear(const int dims[4], const void* links_in, void* links_out, double rho, double epsilon,
                         int steps, void* cuda_stream);

/* Last error message of the context ("" if none); never NULL.  Passing NULL
 * returns the message of the last failed ov_create or ov_wilson_noalloc call
 * on this thread. */
const char* ov_last_error(const ov_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* OVERLAP_GB300_H */
