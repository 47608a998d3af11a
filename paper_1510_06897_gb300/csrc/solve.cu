// CG on the normal equations D^dagger D x = D^dagger b, or on the chiral-sector
// operator, with the inner solver in the context's precision inside an FP64
// defect correction on the true residual.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace ov {

// CG on D^dagger D e = r0 for each RHS, with the operator of instance I;
// vectors in I.pv.  Stops when |r|/|r0| <= tol for every RHS (iterated
// residual).  Returns the iteration count in *iters.
ov_status cg_inner(ov_ctx* c, Inst& I, const void* r0, void* e, int nrhs, double mu, double tol, int maxit,
                   int* iters, int chirality) {
  const int64_t V = c->g.V;
  const size_t vb = I.vbytes(V) * nrhs, v1 = I.vbytes(V);
  OV_CK(I.cx.ensure(vb));
  OV_CK(I.cr.ensure(vb));
  OV_CK(I.cp.ensure(vb));
  OV_CK(I.cq.ensure(vb));
  OV_TRY(ensure_work(c, I, nrhs));
  OV_CK(cudaMemsetAsync(e, 0, vb, c->st));
  OV_CK(cudaMemcpyAsync(I.cr.p, r0, vb, cudaMemcpyDeviceToDevice, c->st));
  OV_CK(cudaMemcpyAsync(I.cp.p, r0, vb, cudaMemcpyDeviceToDevice, c->st));
  std::vector<double> rr(nrhs), rr0(nrhs);
  std::vector<char> done(nrhs, 0);
  for (int r = 0; r < nrhs; ++r) {
    OV_TRY(norm2(c, I.pv, I.cr.c() + r * v1, V, &rr[r]));
    rr0[r] = rr[r];
    if (rr0[r] == 0.0) done[r] = 1;
  }
  const bool is16 = (I.p == OP_F16 || I.p == OP_B16);
  int it = 0;
  for (; it < maxit; ++it) {
    bool all = true;
    for (int r = 0; r < nrhs; ++r) all = all && done[r];
    if (all) break;
    double rmax = 0.0;
    for (int r = 0; r < nrhs; ++r)
      if (!done[r]) rmax = std::max(rmax, std::sqrt(rr[r]));
    // keep 16-bit recurrence vectors at O(1) per component
    const double scale = is16 ? std::sqrt(24.0 * (double)V) / rmax : 1.0;
    OV_TRY(op_apply(c, I, I.cp.p, I.cq.p, nrhs, mu, scale, chirality));
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      double2 pq;
      OV_TRY(dots(c, I.pv, I.cp.c() + r * v1, I.cq.c() + r * v1, V, &pq));
      if (!(pq.x > 0.0) || !std::isfinite(pq.x))
        return fail(c, OV_ERR_NOT_CONVERGED, "CG breakdown: p^dagger A p <= 0 or not finite");
      const double alpha = rr[r] / pq.x;
      launch_cg_update_xr(I.pv, static_cast<char*>(e) + r * v1, I.cr.c() + r * v1, I.cp.c() + r * v1,
                          I.cq.c() + r * v1, alpha, V, 1, c->d_partial.as<double2>(), c->st);
      OV_TRY(launched(c));
      double2 rn;
      OV_TRY(read_reduced(c, c->d_partial.as<double2>(), 1, &rn));
      const double beta = rn.x / rr[r];
      rr[r] = rn.x;
      if (!std::isfinite(rn.x)) return fail(c, OV_ERR_NOT_CONVERGED, "CG residual not finite");
      if (std::sqrt(rr[r]) <= tol * std::sqrt(rr0[r])) {
        done[r] = 1;
        continue;
      }
      launch_cg_update_p(I.pv, I.cp.c() + r * v1, I.cr.c() + r * v1, beta, V, 1, c->st);
      OV_TRY(launched(c));
    }
  }
  *iters = it;
  for (int r = 0; r < nrhs; ++r)
    if (!done[r]) return OV_ERR_NOT_CONVERGED;  // caller decides; no message overwrite
  return OV_OK;
}


// CG on D^dagger D x = D^dagger b (chirality 0) or on the chiral-sector
// operator A x = P b (chirality +-1), FP64 defect correction around the
// inner solver of the context's precision.
ov_status solve_core(ov_ctx* c, double mu, int chirality, double tol, int maxit, const void* b, void* x, int nrhs,
                     ov_dtype dt, int* iters, double* true_rel_resid) {
  if (!c) return OV_ERR_INVALID;
  if (!b || !x) return fail(c, OV_ERR_INVALID, "null vector");
  if (!std::isfinite(mu) || !(tol > 0.0) || maxit < 1)
    return fail(c, OV_ERR_INVALID, "need finite mu, tol > 0, maxit >= 1");
  OV_TRY(check_dtype(c, nrhs, dt));
  if (!c->configured) return fail(c, OV_ERR_STATE, "sign(K) not configured: call ov_sign_config first");
  c->stats.inner_iterations = 0;
  c->stats.outer_iterations = 0;
  c->res_history.clear();
  Inst& H = c->hi;
  // inner solver: FP64 itself, or the context-precision operator
  Inst& I = (c->prec == OV_FP64) ? c->hi : c->lo;
  const int64_t V = c->g.V;
  const size_t v1 = H.vbytes(V), vb = v1 * nrhs;
  const size_t iv1 = I.vbytes(V);
  OV_TRY(ensure_work(c, H, nrhs));
  OV_TRY(ensure_work(c, I, nrhs));
  OV_CK(c->o_x.ensure(vb));
  OV_CK(c->o_r.ensure(vb));
  OV_CK(c->o_rhs.ensure(vb));
  OV_CK(c->o_q.ensure(vb));
  OV_CK(I.cx.ensure(iv1 * nrhs));
  // rhs = D^dagger b with the FP64 operator, or P b (the FP64 layout keeps
  // spinor component 3 spin + colour in chunk k: spins 2, 3 are chunks 6..11)
  OV_TRY(pack_input(c, H, b, nrhs, dt, H.xin.p));
  if (chirality == 0) {
    OV_TRY(sign_core(c, H, H.xin.p, c->o_rhs.p, nrhs, K_OVL_DAG, mu, 1.0));
  } else {
    OV_CK(cudaMemcpyAsync(c->o_rhs.p, H.xin.p, vb, cudaMemcpyDeviceToDevice, c->st));
    const size_t half = v1 / 2;
    for (int r = 0; r < nrhs; ++r)
      OV_CK(cudaMemsetAsync(c->o_rhs.c() + r * v1 + (chirality > 0 ? half : 0), 0, half, c->st));
  }
  std::vector<double> rhs_n(nrhs), res(nrhs), rn(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    OV_TRY(norm2(c, OP_F64, c->o_rhs.c() + r * v1, V, &rhs_n[r]));
    rhs_n[r] = std::sqrt(rhs_n[r]);
    res[r] = rhs_n[r] > 0 ? 1.0 : 0.0;
    rn[r] = rhs_n[r];
  }
  OV_CK(cudaMemsetAsync(c->o_x.p, 0, vb, c->st));
  OV_CK(cudaMemcpyAsync(c->o_r.p, c->o_rhs.p, vb, cudaMemcpyDeviceToDevice, c->st));

  // Defect correction: r = rhs - A x (FP64), solve A e = r / |r| with inner CG,
  // x += |r| e, recompute r.  With an FP64 inner solver the first pass usually
  // meets tol already; the loop then only confirms it.
  const int max_outer = (c->prec == OV_FP64) ? 4 : c->max_outer;
  int total = 0;
  bool ok = false;
  for (int outer = 0; outer < max_outer; ++outer) {
    double worst = 0;
    for (double v : res) worst = std::max(worst, v);
    if (worst <= tol) {
      ok = true;
      break;
    }
    if (total >= maxit) break;
    for (int r = 0; r < nrhs; ++r) {
      launch_convert(OP_F64, I.pv, c->o_r.c() + r * v1, I.xin.c() + r * iv1, V, 1, rn[r] > 0 ? 1.0 / rn[r] : 0.0,
                     0, c->st);
      OV_TRY(launched(c));
    }
    double inner = 0.5 * tol / worst;
    if (c->prec != OV_FP64) inner = std::max(inner, c->inner_tol);
    inner = std::min(inner, 0.5);
    int it = 0;
    ov_status s = cg_inner(c, I, I.xin.p, I.cx.p, nrhs, mu, inner, maxit - total, &it, chirality);
    total += it;
    if (s != OV_OK && s != OV_ERR_NOT_CONVERGED) return s;
    for (int r = 0; r < nrhs; ++r) {
      launch_convert(I.pv, OP_F64, I.cx.c() + r * iv1, c->o_x.c() + r * v1, V, 1, rn[r], 1, c->st);
      OV_TRY(launched(c));
    }
    c->stats.outer_iterations++;
    // true residual with the FP64 operator
    OV_TRY(op_apply(c, H, c->o_x.p, c->o_q.p, nrhs, mu, 1.0, chirality));
    launch_axpby(OP_F64, 1.0, c->o_rhs.p, -1.0, c->o_q.p, c->o_r.p, V, nrhs, c->st);
    OV_TRY(launched(c));
    for (int r = 0; r < nrhs; ++r) {
      double n2;
      OV_TRY(norm2(c, OP_F64, c->o_r.c() + r * v1, V, &n2));
      rn[r] = std::sqrt(n2);
      res[r] = rhs_n[r] > 0 ? rn[r] / rhs_n[r] : 0.0;
    }
    c->res_history.push_back(*std::max_element(res.begin(), res.end()));
  }
  if (!ok) {
    double worst = 0;
    for (double v : res) worst = std::max(worst, v);
    ok = worst <= tol;
  }
  c->stats.inner_iterations = total;
  OV_TRY(unpack_output(c, H, c->o_x.p, x, nrhs, dt));
  if (iters) *iters = total;
  double mx = 0;
  for (double v : res) mx = std::max(mx, v);
  if (true_rel_resid) *true_rel_resid = mx;
  if (!ok) return fail(c, OV_ERR_NOT_CONVERGED, "solver stopped before reaching tol");
  return OV_OK;
}

}  // namespace ov

extern "C" {

ov_status ov_set_solver_params(ov_ctx* c, double inner_tol, int max_outer) {
  if (!c) return OV_ERR_INVALID;
  if (!(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
    return fail(c, OV_ERR_INVALID, "need 0 < inner_tol < 1 and max_outer >= 1");
  c->inner_tol = inner_tol;
  c->max_outer = max_outer;
  return OV_OK;
}

ov_status ov_solve(ov_ctx* c, double mu, double tol, int maxit, const void* b, void* x, int nrhs, ov_dtype dt,
                   int* iters, double* true_rel_resid) {
  return solve_core(c, mu, 0, tol, maxit, b, x, nrhs, dt, iters, true_rel_resid);
}

ov_status ov_solve_chiral(ov_ctx* c, double mu, int chirality, double tol, int maxit, const void* b, void* x,
                          int nrhs, ov_dtype dt, int* iters, double* true_rel_resid) {
  if (!c) return OV_ERR_INVALID;
  if (chirality != 1 && chirality != -1) return fail(c, OV_ERR_INVALID, "chirality must be +1 or -1");
  if (!(std::fabs(mu) < 1.0)) return fail(c, OV_ERR_INVALID, "need |mu| < 1 (positive definite sector operator)");
  return solve_core(c, mu, chirality, tol, maxit, b, x, nrhs, dt, iters, true_rel_resid);
}

}  // extern "C"
