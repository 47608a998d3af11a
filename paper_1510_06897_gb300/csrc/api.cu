// C ABI of the overlap library: context creation and destruction, argument
// checks and the entry points for D_W, K, sign(K), D[mu], statistics and
// profiling.  The sign(K) driver lives in sign.cu, the solvers in solve.cu,
// the stencil tuning in tune.cu and the shared helpers in ctx.cu; all
// arithmetic runs in the kernels of dslash*.cu / blas.cu / eigs.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace ov;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace ov {
// Message returned by ov_last_error(NULL) on this thread (context-free calls).
void set_thread_error(const std::string& msg) { g_create_error = msg; }
}  // namespace ov

// ===========================================================================
// C ABI

extern "C" {

ov_status ov_create(ov_ctx** ctx, const int dims[4], const void* links, ov_prec prec, double m_w, int antiperiodic_t,
                    void* cuda_stream) {
  g_create_error.clear();
  if (!ctx || !dims || !links) {
    g_create_error = "ov_create: null argument";
    return OV_ERR_INVALID;
  }
  *ctx = nullptr;
  int64_t V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2) {
      g_create_error = "ov_create: every lattice extent must be >= 2";
      return OV_ERR_INVALID;
    }
    V *= dims[i];
  }
  if (V > (int64_t(1) << 31) / 16) {
    g_create_error = "ov_create: lattice too large";
    return OV_ERR_INVALID;
  }
  if ((int64_t)dims[2] * dims[3] > 65535) {  // the stencil grid's y dimension is one (z, t) slice each
    g_create_error = "ov_create: Lz * Lt must be <= 65535";
    return OV_ERR_INVALID;
  }
  if (prec < OV_FP64 || prec > OV_MIXED_BF16) {
    g_create_error = "ov_create: unknown precision";
    return OV_ERR_INVALID;
  }
  if (!std::isfinite(m_w)) {
    g_create_error = "ov_create: m_w not finite";
    return OV_ERR_INVALID;
  }
  ov_ctx* c = new ov_ctx();
  for (int i = 0; i < 4; ++i) c->g.L[i] = dims[i];
  c->g.V = V;
  c->g.antiperiodic_t = antiperiodic_t ? 1 : 0;
  c->m_w = m_w;
  c->prec = prec;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  if (const char* chk = std::getenv("OV_CHECKS")) c->checks = std::atoi(chk) != 0;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (c->num_sms <= 0) c->num_sms = 148;
  }
  // flag of the slab stencil (without it the slab kernel is not used)
  if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_stencil_err), sizeof(int), cudaHostAllocMapped) == cudaSuccess) {
    *c->h_stencil_err = 0;
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_stencil_err), c->h_stencil_err, 0) != cudaSuccess)
      c->d_stencil_err = nullptr;
  } else {
    c->h_stencil_err = nullptr;
  }
  cudaGetLastError();
  const void* dl = nullptr;
  ov_status s = stage_in(c, c->stage_links, links, (size_t)V * 4 * 9 * 16, &dl);
  if (s == OV_OK) s = init_inst(c, c->hi, OP_F64, dl);
  if (s == OV_OK && prec != OV_FP64) {
    const OpPrec lp = prec == OV_FP32 ? OP_F32 : prec == OV_MIXED_FP16 ? OP_F16 : OP_B16;
    s = init_inst(c, c->lo, lp, dl);
  }
  if (s == OV_OK) {
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) s = fail(c, OV_ERR_CUDA, cudaGetErrorString(e));
  }
  c->stage_links.release();
  if (s != OV_OK) {
    g_create_error = c->err;
    ov_destroy(c);
    return s;
  }
  *ctx = c;
  return OV_OK;
}

ov_status ov_destroy(ov_ctx* c) {
  if (!c) return OV_OK;
  cudaStreamSynchronize(c->st);
  if (c->l2_pinned) {
    if (l2_window().base == c->lo.links.p) l2_window() = L2Window{};
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
  }
  c->hi.release();
  c->lo.release();
  c->mid.release();
  c->gw.release();
  for (cudaEvent_t ev : c->evs) cudaEventDestroy(ev);
  for (DevBuf* b : {&c->d_sgn, &c->d_c, &c->d_partial, &c->d_scalars, &c->d_gram, &c->d_err, &c->d_never, &c->stage_in, &c->stage_out, &c->stage_links,
                    &c->o_x, &c->o_r, &c->o_rhs, &c->o_q})
    b->release();
  if (c->h_scalars) cudaFreeHost(c->h_scalars);
  if (c->h_stencil_err) cudaFreeHost(c->h_stencil_err);
  delete c;
  return OV_OK;
}

static ov_status apply_stencil(ov_ctx* c, const void* in, void* out, int nrhs, ov_dtype dt, int wilson) {
  if (!c) return OV_ERR_INVALID;
  if (!in || !out) return fail(c, OV_ERR_INVALID, "null vector");
  OV_TRY(check_dtype(c, nrhs, dt));
  Inst& I = c->op();
  OV_TRY(ensure_work(c, I, nrhs));
  OV_TRY(pack_input(c, I, in, nrhs, dt, I.xin.p));
  const void* src = I.xin.p;
  if (I.p != I.pv) {
    launch_convert(I.pv, I.p, I.xin.p, I.perp.p, c->g.V, nrhs, 1.0, 0, c->st);
    OV_TRY(launched(c));
    src = I.perp.p;
  }
  EpiArgs e;
  e.wilson = wilson;
  e.m_w = c->m_w;
  OV_TRY(dslash(c, I, I.pv, src, I.xout.p, e, nrhs));
  return unpack_output(c, I, I.xout.p, out, nrhs, dt);
}

ov_status ov_wilson(ov_ctx* c, const void* in, void* out, int nrhs, ov_dtype dt) {
  return apply_stencil(c, in, out, nrhs, dt, 1);
}

ov_status ov_kernel(ov_ctx* c, const void* in, void* out, int nrhs, ov_dtype dt) {
  return apply_stencil(c, in, out, nrhs, dt, 0);
}

ov_status ov_sign_config(ov_ctx* c, int order, double lo, double hi, const double* evals, const void* evecs,
                         int n_ev) {
  if (!c) return OV_ERR_INVALID;
  if (order < 1) return fail(c, OV_ERR_INVALID, "Chebyshev order must be >= 1");
  if (!(lo > 0.0) || !(hi > lo) || !std::isfinite(hi)) return fail(c, OV_ERR_INVALID, "need 0 < lo < hi");
  if (n_ev < 0) return fail(c, OV_ERR_INVALID, "n_ev must be >= 0");
  if (n_ev > 0 && (!evals || !evecs)) return fail(c, OV_ERR_INVALID, "n_ev > 0 needs evals and evecs");
  for (int i = 0; i < n_ev; ++i)
    if (!std::isfinite(evals[i])) return fail(c, OV_ERR_INVALID, "eigenvalue not finite");
  c->configured = false;
  c->order = order;
  c->a = lo;
  c->b = hi;
  c->coef = chebyshev_coefficients(order, lo, hi);
  c->n_ev = n_ev;
  c->evals.assign(evals, evals + n_ev);
  c->sgn.resize(n_ev);
  for (int i = 0; i < n_ev; ++i) c->sgn[i] = evals[i] >= 0.0 ? 1.0 : -1.0;
  OV_CK(c->d_sgn.ensure(sizeof(double) * std::max(1, n_ev)));
  if (n_ev > 0) {
    OV_CK(cudaMemcpyAsync(c->d_sgn.p, c->sgn.data(), sizeof(double) * n_ev, cudaMemcpyHostToDevice, c->st));
    const size_t ib = iface_bytes(c->g, n_ev, OV_C128);
    const void* de;
    OV_TRY(stage_in(c, c->stage_in, evecs, ib, &de));
    for (Inst* I : {&c->hi, &c->lo, &c->mid}) {
      if (!I->active) continue;
      OV_CK(I->evecs.ensure(I->vbytes(c->g.V) * n_ev));
      launch_pack_spinor(I->pv, IF_C128, c->g, de, I->evecs.p, n_ev, 1.0, 0, c->st);
      OV_TRY(launched(c));
    }
    c->stage_in.release();
  }
  OV_CK(cudaStreamSynchronize(c->st));
  c->configured = true;
  return OV_OK;
}

ov_status ov_sign_apply(ov_ctx* c, const void* in, void* out, int nrhs, ov_dtype dt) {
  if (!c) return OV_ERR_INVALID;
  if (!in || !out) return fail(c, OV_ERR_INVALID, "null vector");
  OV_TRY(check_dtype(c, nrhs, dt));
  if (!c->configured) return fail(c, OV_ERR_STATE, "sign(K) not configured: call ov_sign_config first");
  Inst& I = c->op();
  OV_TRY(ensure_work(c, I, nrhs));
  OV_TRY(pack_input(c, I, in, nrhs, dt, I.xin.p));
  OV_TRY(sign_core(c, I, I.xin.p, I.xout.p, nrhs, K_SIGN, 0.0, 1.0));
  return unpack_output(c, I, I.xout.p, out, nrhs, dt);
}

ov_status ov_sign(ov_ctx* c, int order, double lo, double hi, const double* evals, const void* evecs, int n_ev,
                  const void* in, void* out, int nrhs, ov_dtype dt) {
  OV_TRY(ov_sign_config(c, order, lo, hi, evals, evecs, n_ev));
  return ov_sign_apply(c, in, out, nrhs, dt);
}

ov_status ov_overlap(ov_ctx* c, double mu, int dagger, const void* in, void* out, int nrhs, ov_dtype dt) {
  if (!c) return OV_ERR_INVALID;
  if (!in || !out) return fail(c, OV_ERR_INVALID, "null vector");
  if (!std::isfinite(mu)) return fail(c, OV_ERR_INVALID, "mu not finite");
  OV_TRY(check_dtype(c, nrhs, dt));
  if (!c->configured) return fail(c, OV_ERR_STATE, "sign(K) not configured: call ov_sign_config first");
  Inst& I = c->op();
  OV_TRY(ensure_work(c, I, nrhs));
  OV_TRY(pack_input(c, I, in, nrhs, dt, I.xin.p));
  OV_TRY(sign_core(c, I, I.xin.p, I.xout.p, nrhs, dagger ? K_OVL_DAG : K_OVL, mu, 1.0));
  return unpack_output(c, I, I.xout.p, out, nrhs, dt);
}

ov_status ov_get_stats(const ov_ctx* c, ov_stats* out) {
  if (!c || !out) return OV_ERR_INVALID;
  *out = c->stats;
  const Inst& I = (c->prec == OV_FP64) ? c->hi : c->lo;
  out->stencil_tpb = I.cfg.tpb;
  out->stencil_minb = I.cfg.minb;
  out->stencil_lrec = (I.p == OP_F64) ? 18 : I.cfg.lrec;
  out->stencil_slab = I.cfg.slab;
  out->stencil_async = I.cfg.async;
  out->stencil_brick = I.cfg.brick;
  return OV_OK;
}

ov_status ov_set_profiling(ov_ctx* c, int on) {
  if (!c) return OV_ERR_INVALID;
  if (!on && c->ev_used) {
    OV_CK(cudaStreamSynchronize(c->st));
    prof_collect(c);
  }
  c->prof = (on == 2) ? 2 : (on ? 1 : 0);
  return OV_OK;
}

ov_status ov_get_residual_history(const ov_ctx* c, double* out, int max_len, int* len) {
  if (!c || max_len < 0 || (max_len > 0 && !out)) return OV_ERR_INVALID;
  const int n = (int)c->res_history.size();
  for (int i = 0; i < std::min(n, max_len); ++i) out[i] = c->res_history[i];
  if (len) *len = n;
  return OV_OK;
}

ov_status ov_test_wait_expiry(ov_ctx* c, long long cycles) {
  if (!c) return OV_ERR_INVALID;
  if (cycles > 0 && c->d_never.p == nullptr) {  // the flag nothing sets
    OV_CK(c->d_never.ensure(sizeof(int)));
    OV_CK(cudaMemsetAsync(c->d_never.p, 0, sizeof(int), c->st));
    OV_CK(cudaStreamSynchronize(c->st));
  }
  c->stall_cycles = cycles > 0 ? cycles : 0;
  return OV_OK;
}

ov_status ov_set_checks(ov_ctx* c, int on) {
  if (!c) return OV_ERR_INVALID;
  c->checks = on != 0;
  return OV_OK;
}

ov_status ov_reset_stats(ov_ctx* c) {
  if (!c) return OV_ERR_INVALID;
  c->stats = ov_stats{};
  return OV_OK;
}

const char* ov_last_error(const ov_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

}  // extern "C"

