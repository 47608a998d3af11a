// Context of the C ABI and the host-side helpers shared by the drivers
// (api.cu: entry points; sign.cu: sign(K) and the overlap operators; solve.cu:
// solvers; tune.cu: stencil shapes; ctx.cu: these helpers; eigs_host.cu:
// eigensolver; grad_host.cu: adjoint).  Not part of the public interface.
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include "../../include/overlap.h"
#include "internal.h"

namespace ov {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
  char* c() const { return static_cast<char*>(p); }
};

// Device vectors of ov_sign_poly_quad / ov_sign_poly_grad, kept between calls
// so that repeated gradients (one per molecular-dynamics step) allocate
// nothing; ov_set_grad_memory and ov_destroy release them.
struct GradWork {
  DevBuf xchi, rot, ck, segb, segt, bbar, tbar, gvec, gbar, zero, t, G, keep;
  void release() {
    for (DevBuf* b : {&xchi, &rot, &ck, &segb, &segt, &bbar, &tbar, &gvec, &gbar, &zero, &t, &G, &keep}) b->release();
  }
};

// One operator instance: links, eigenvectors and work vectors in one precision.
struct Inst {
  OpPrec p = OP_F64;   // link / recurrence storage
  OpPrec pv = OP_F64;  // vector storage: deflation, assembly, solver vectors
  bool active = false;
  DslashCfg cfg;  // stencil launch shape / link layout for one RHS (autotuned at create)
  std::vector<std::pair<int, DslashCfg>> cfg_batch;  // tuned shapes for nrhs > 1
  DevBuf links, evecs;
  DevBuf xin, xout, d, tmp;          // pv
  DevBuf perp, t, bA, bB;            // p
  DevBuf cx, cr, cp, cq;             // pv: inner CG
  DevBuf sv, svt, sw, sdh, sdt, sx;  // pv: SUMR
  DevBuf gr, grhs, gu, gc;           // pv: GCR residual, inner right-hand side, directions u_i and c_i = D u_i
  size_t vbytes(int64_t V) const { return (size_t)spinor_bytes_per_site(pv) * V; }
  size_t pbytes(int64_t V) const { return (size_t)spinor_bytes_per_site(p) * V; }
  void release() {
    for (DevBuf* b : {&links, &evecs, &xin, &xout, &d, &tmp, &perp, &t, &bA, &bB, &cx, &cr, &cp, &cq, &sv, &svt, &sw,
                      &sdh, &sdt, &sx, &gr, &grhs, &gu, &gc})
      b->release();
  }
};

// K_CHI_P / K_CHI_M: the chiral-sector normal operator (input of that chirality):
// out = 1/4 [(1+mu)^2 + (1-mu)^2] in +- 1/2 (1 - mu^2) P sign(K) in
enum Kind { K_SIGN, K_OVL, K_OVL_DAG, K_CHI_P, K_CHI_M };

}  // namespace ov

using namespace ov;

struct ov_ctx {
  LatticeH g{};
  double m_w = 1.5;
  cudaStream_t st = nullptr;
  ov_prec prec = OV_FP64;
  Inst hi;  // FP64 operator (always)
  Inst lo;  // operator in the context precision when it is not FP64
  Inst mid;  // FP32 operator beside a 16-bit one (ov_enable_fp32_operator): the GCR level of GMRESR
  // sign configuration
  bool configured = false;
  int order = 0;
  double a = 0, b = 0;
  std::vector<double> coef;
  int n_ev = 0;
  std::vector<double> evals, sgn;
  DevBuf d_sgn, d_c, d_partial, d_scalars, d_gram, d_err;
  int num_sms = 0;
  bool l2_pinned = false;  // this context set the persisting-L2 window over its links
  DevBuf stage_in, stage_out, stage_links;
  DevBuf o_x, o_r, o_rhs, o_q;  // FP64 outer-solver vectors
  double* h_scalars = nullptr;  // pinned
  int h_scalars_n = 0;
  int* h_stencil_err = nullptr;  // mapped pinned flag of the slab stencil (device view d_stencil_err)
  int* d_stencil_err = nullptr;
  // output checks (ov_set_checks / OV_CHECKS=1): every vector output is
  // scanned for NaN / Inf before it is handed back
  bool checks = false;
  // testing (ov_test_wait_expiry): > 0 makes the pipeline waits of the
  // kernels that wait on their own asynchronous work first wait this many
  // cycles on d_never, a device flag that nothing sets, and report expiry
  long long stall_cycles = 0;
  DevBuf d_never;
  // solver controls
  double inner_tol = 1e-5;
  int max_outer = 30;
  // GMRESR: inner SUMR order (0: automatic), tolerance, products per inner
  // solve, GCR directions kept; the relaxed coefficients and what they were made for
  int gm_order = 0;
  double gm_tol = 0.1;
  int gm_maxit = 1000;
  int gm_dirs = 12;
  // GCR level of GMRESR on an FP32 copy of the operator for 16-bit contexts
  // (built from the FP64 links on first use unless switched off)
  bool gm_fp32 = true;
  // gradient (ov_set_grad_memory): device bytes the recurrence terms may
  // occupy so that none is recomputed; < 0: half the free memory at the call
  long long grad_mem = -1;
  GradWork gw;
  std::vector<double> coef_relaxed;
  double relaxed_key[4] = {0, 0, 0, 0};
  ov_stats stats{};
  std::vector<double> res_history;  // largest true relative residual after each FP64 pass of the last solve
  std::string err;
  // stencil profiling (ov_set_profiling): 1 = an event pair around every
  // stencil launch, 2 = one pair around each run of back-to-back stencil
  // launches (the recurrence), with the number of launches it holds
  int prof = 0;
  std::vector<cudaEvent_t> evs;
  std::vector<int> ev_count;  // stencil launches inside each recorded pair
  size_t ev_used = 0;

  Inst& op() { return prec == OV_FP64 ? hi : lo; }
};


namespace ov {

ov_status fail(ov_ctx* c, ov_status s, const std::string& msg);
ov_status launched(ov_ctx* c, int n = 1);
ov_status stage_in(ov_ctx* c, DevBuf& buf, const void* p, size_t bytes, const void** out);
ov_status stage_out(ov_ctx* c, void* p, size_t bytes, void** out, bool* staged);
ov_status finish_out(ov_ctx* c, void* host, size_t bytes, bool staged);
size_t iface_bytes(const LatticeH& g, int nrhs, ov_dtype dt);
ov_status read_reduced(ov_ctx* c, const double2* partial, int n, double2* out);
ov_status ensure_work(ov_ctx* c, Inst& I, int nrhs);
ov_status norm2(ov_ctx* c, OpPrec p, const void* a, int64_t V, double* out);
ov_status dots(ov_ctx* c, OpPrec p, const void* a, const void* b, int64_t V, double2* out);
std::vector<double> chebyshev_coefficients(int order, double a, double b);
ov_status pack_input(ov_ctx* c, Inst& I, const void* in, int nrhs, ov_dtype dt, void* dst);
ov_status unpack_output(ov_ctx* c, Inst& I, const void* src, void* out, int nrhs, ov_dtype dt);
ov_status check_dtype(ov_ctx* c, int nrhs, ov_dtype dt);
// launch the stencil of instance I (counted, profiled when enabled)
ov_status dslash(ov_ctx* c, Inst& I, OpPrec out_prec, const void* in, void* out, const EpiArgs& e, int nrhs);
// fold completed profiling event pairs into the stats (call after a stream sync)
void prof_collect(ov_ctx* c);
// profiling mode 2: open / close an event pair around n back-to-back stencil launches
ov_status prof_open(ov_ctx* c);
ov_status prof_close(ov_ctx* c, int n);
// out (storage I.p) = stencil epilogue of K applied to `in` (see EpiArgs)
ov_status k_step(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, const EpiArgs& e);
// cf: Chebyshev coefficients to use instead of the configured ones (a
// lower-order polynomial on the same interval), or null
ov_status sign_core(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, Kind kind, double mu, double scale,
                    const std::vector<double>* cf = nullptr);
// max over [a^2, b^2] of |sqrt(y) f_N(y) - 1| for the coefficients cf (sign.cu)
double chebyshev_sign_error(const std::vector<double>& cf, double a, double b);
ov_status normal_apply(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, double mu, double scale);
// D^dagger D (chirality 0) or the chiral-sector operator (chirality +-1)
ov_status op_apply(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, double mu, double scale, int chirality);
// operator instance in storage p: links packed from the complex128 interface
// layout, stencil shape tuned, 16-bit links marked persisting in L2 (tune.cu)
ov_status init_inst(ov_ctx* c, Inst& I, OpPrec p, const void* links_dev);
// stencil shape for nrhs right-hand sides, tuned on first use (tune.cu)
ov_status batch_cfg(ov_ctx* c, Inst& I, int nrhs, DslashCfg* out);

}  // namespace ov

#define OV_CK(call)                                                                             \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return ov::fail(c, e_ == cudaErrorMemoryAllocation ? OV_ERR_NOMEM : OV_ERR_CUDA,          \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

#define OV_TRY(expr)              \
  do {                            \
    ov_status s_ = (expr);        \
    if (s_ != OV_OK) return s_;   \
  } while (0)
