// GMRESR for D[mu] x = b (Sec. 2: recursive GMRES whose preconditioner is a
// low-accuracy shifted-unitary minimal residual solve with a relaxed sign
// function), with the mixed-precision defect correction of the CG solver:
//
//   FP64 defect correction on D[mu] (accurate sign, FP64 operator)
//     GCR on D[mu] in the context precision (accurate order)
//       SUMR on U = gamma5 S in the context precision (relaxed order)
//
// SUMR.  D[mu] = (1 - mu)/2 (U - zeta), zeta = -(1 + mu)/(1 - mu), so
// D x = b is (U - zeta) x = 2 b / (1 - mu).  The minimal residual iterate
// over the Krylov space of U comes from the Szego recursion of the
// orthonormal polynomials phi_j of U (one product with U per step):
//   m = <v~_j, U v_j>,  v_{j+1} = (U v_j - m v~_j) / rho_j,  v~_{j+1} = (v~_j - conj(m) U v_j) / rho~_j,
//   D_{j+1} = (v_j + zeta D_j - m D~_j) / rho_j,  D~_{j+1} = (D~_j - conj(m) (v_j + zeta D_j)) / rho~_j,
//   phi_{j+1}(zeta) = (zeta phi_j - m phi^*_j) / rho_j,  phi^*_{j+1}(zeta) = (phi^*_j - conj(m) zeta phi_j) / rho~_j,
//   x_k = -(|b'| / s_k) sum_j conj(phi_j(zeta)) D_j,  s_k = sum_j |phi_j(zeta)|^2,
// with rho_j, rho~_j the computed norms of the new pair (for exactly unitary
// U both equal sqrt(1 - |m|^2); normalising by the computed norms keeps the
// recursion stable when U = gamma5 P(K) is unitary only to the Chebyshev
// error).  The residual estimate is 1/sqrt(s_k).  On the device the stored
// vectors carry the previous step's divisors (lazy normalisation), so one
// fused kernel per step updates all six vectors and returns the two norms.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace ov {

using zc = std::complex<double>;

static double2 d2(zc z) { return make_double2(z.real(), z.imag()); }

// Relaxed coefficient set for the inner solves: gm_order if set, else the
// smallest order whose sign error on [a, b] is <= 1e-2; never above the
// configured order.
static ov_status relaxed_coefficients(ov_ctx* c) {
  const double key[4] = {(double)c->gm_order, c->a, c->b, (double)c->order};
  if (!c->coef_relaxed.empty() && std::memcmp(key, c->relaxed_key, sizeof(key)) == 0) return OV_OK;
  int n = c->order;
  if (c->gm_order > 0) {
    n = std::min(c->gm_order, c->order);
  } else {
    int lo = 1, hi = c->order;  // bisection: the error of the interpolant falls with the order
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (chebyshev_sign_error(chebyshev_coefficients(mid, c->a, c->b), c->a, c->b) <= 1e-2)
        hi = mid;
      else
        lo = mid + 1;
    }
    n = lo;
  }
  c->coef_relaxed = chebyshev_coefficients(n, c->a, c->b);
  std::memcpy(c->relaxed_key, key, sizeof(key));
  return OV_OK;
}

static ov_status ensure_sumr(ov_ctx* c, Inst& I, int nrhs) {
  const size_t vb = I.vbytes(c->g.V) * nrhs;
  for (DevBuf* b : {&I.sv, &I.svt, &I.sw, &I.sdh, &I.sdt, &I.sx}) OV_CK(b->ensure(vb));
  return ensure_work(c, I, nrhs);
}

// SUMR for D[mu] x = b on nrhs right-hand sides (storage I.pv), sign(K) of
// instance I with coefficients cf.  Each RHS stops when its estimate
// 1/sqrt(s) <= tol, after maxit products with U, or when the new Krylov
// pair has (numerically) zero norm (invariant subspace).  x may alias
// nothing else.  *iters: products with U (all RHS advance together);
// *est: the largest final estimate.
ov_status sumr_core(ov_ctx* c, Inst& I, const std::vector<double>& cf, double mu, const void* b, void* x, int nrhs,
                    double tol, int maxit, int* iters, double* est) {
  const int64_t V = c->g.V;
  const size_t v1 = I.vbytes(V);
  OV_TRY(ensure_sumr(c, I, nrhs));
  const double zeta = -(1.0 + mu) / (1.0 - mu);
  const bool is16 = (I.p == OP_F16 || I.p == OP_B16);
  std::vector<double> nb(nrhs), av(nrhs, 1.0), at(nrhs, 1.0), s(nrhs, 1.0);
  std::vector<zc> phi(nrhs, 1.0), phis(nrhs, 1.0), cx(nrhs, 0.0);
  std::vector<char> done(nrhs, 0);
  // v_0 = v~_0 = b / |b| (b' = 2 b / (1 - mu) has the same direction)
  for (int r = 0; r < nrhs; ++r) {
    double n2;
    OV_TRY(norm2(c, I.pv, static_cast<const char*>(b) + r * v1, V, &n2));
    nb[r] = std::sqrt(n2);
    if (!std::isfinite(nb[r])) return fail(c, OV_ERR_INVALID, "SUMR: right-hand side not finite");
    done[r] = !(nb[r] > 0.0) || tol >= 1.0;
    launch_axpby(I.pv, nb[r] > 0.0 ? 1.0 / nb[r] : 0.0, static_cast<const char*>(b) + r * v1, 0.0, nullptr,
                 I.sv.c() + r * v1, V, 1, c->st);
    OV_TRY(launched(c));
  }
  OV_CK(cudaMemcpyAsync(I.svt.p, I.sv.p, v1 * nrhs, cudaMemcpyDeviceToDevice, c->st));
  for (DevBuf* z : {&I.sdh, &I.sdt, &I.sx}) OV_CK(cudaMemsetAsync(z->p, 0, v1 * nrhs, c->st));
  int it = 0;
  for (; it < maxit; ++it) {
    bool all = true;
    double vmax = 0.0;
    for (int r = 0; r < nrhs; ++r)
      if (!done[r]) {
        all = false;
        vmax = std::max(vmax, 1.0 / av[r]);
      }
    if (all) break;
    // W = U V = gamma5 S V: D[-1] = gamma5 S; 16-bit recurrences run on O(1) components
    const double scale = is16 ? std::sqrt(24.0 * (double)V) / vmax : 1.0;
    OV_TRY(sign_core(c, I, I.sv.p, I.sw.p, nrhs, K_OVL, -1.0, scale, &cf));
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      double2 tw;
      OV_TRY(dots(c, I.pv, I.svt.c() + r * v1, I.sw.c() + r * v1, V, &tw));
      const zc m = av[r] * at[r] * zc(tw.x, tw.y);
      if (!std::isfinite(m.real()) || !std::isfinite(m.imag()))
        return fail(c, OV_ERR_NOT_CONVERGED, "SUMR: recursion coefficient not finite");
      SumrCoef k;
      k.cx = d2(cx[r]);
      k.av = av[r];
      k.at = at[r];
      k.zv = zeta * av[r];
      k.mt = d2(m * at[r]);
      k.mc = d2(std::conj(m));
      k.mcv = d2(std::conj(m) * av[r]);
      launch_sumr_update(I.pv, I.sv.c() + r * v1, I.svt.c() + r * v1, I.sw.c() + r * v1, I.sdh.c() + r * v1,
                         I.sdt.c() + r * v1, I.sx.c() + r * v1, k, V, c->d_partial.as<double2>(), c->st);
      OV_TRY(launched(c));
      cx[r] = 0.0;  // the deferred term is in X now
      double2 n2;
      OV_TRY(read_reduced(c, c->d_partial.as<double2>(), 1, &n2));
      const double rho = std::sqrt(n2.x), rhot = std::sqrt(n2.y);
      if (!std::isfinite(rho) || !std::isfinite(rhot))
        return fail(c, OV_ERR_NOT_CONVERGED, "SUMR: Krylov vector not finite");
      if (!(std::min(rho, rhot) > 1e-7)) {  // invariant subspace: keep the current iterate
        done[r] = 1;
        continue;
      }
      const zc ph = (zeta * phi[r] - m * phis[r]) / rho;
      phis[r] = (phis[r] - std::conj(m) * zeta * phi[r]) / rhot;
      phi[r] = ph;
      s[r] += std::norm(ph);
      av[r] = 1.0 / rho;
      at[r] = 1.0 / rhot;
      cx[r] = std::conj(ph) * av[r];  // conj(phi_{j+1}) D_{j+1}, added by the next step or below
      if (1.0 / std::sqrt(s[r]) <= tol) done[r] = 1;
    }
  }
  double worst = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    if (cx[r] != 0.0) {
      launch_caxpy(I.pv, d2(cx[r]), I.sdh.c() + r * v1, I.sx.c() + r * v1, V, 1, c->st);
      OV_TRY(launched(c));
    }
    // x = -(|b'| / s) X with |b'| = 2 |b| / (1 - mu)
    const double f = nb[r] > 0.0 ? -2.0 * nb[r] / ((1.0 - mu) * s[r]) : 0.0;
    launch_axpby(I.pv, f, I.sx.c() + r * v1, 0.0, nullptr, static_cast<char*>(x) + r * v1, V, 1, c->st);
    OV_TRY(launched(c));
    if (nb[r] > 0.0) worst = std::max(worst, 1.0 / std::sqrt(s[r]));
  }
  *iters = it;
  *est = worst;
  return OV_OK;
}

// GCR on D[mu] e = r0 with the operator of instance I (its vectors, in
// I.pv, hold the residual and the kept directions), each direction an inner
// SUMR solve with the relaxed coefficients on instance S (S.pv must equal
// I.pv: the SUMR right-hand side and solution live in I's buffers).  Stops
// when the updated residual |r| <= tol |r0| for every RHS, or when the inner
// products reach maxit.  *inner: SUMR products with U; *steps: GCR steps.
static ov_status gcr_core(ov_ctx* c, Inst& I, Inst& S, const void* r0, void* e, int nrhs, double mu, double tol,
                          int maxit, int* inner, int* steps) {
  const int64_t V = c->g.V;
  const size_t v1 = I.vbytes(V), vb = v1 * nrhs;
  const int dirs = c->gm_dirs;
  if (S.pv != I.pv) return fail(c, OV_ERR_INVALID, "GCR and SUMR instances store vectors differently");
  OV_CK(I.gr.ensure(vb));
  OV_CK(I.grhs.ensure(vb));
  OV_CK(I.gu.ensure(vb * dirs));
  OV_CK(I.gc.ensure(vb * dirs));
  OV_TRY(ensure_work(c, I, nrhs));
  OV_TRY(ensure_sumr(c, S, nrhs));
  OV_CK(cudaMemsetAsync(e, 0, vb, c->st));
  OV_CK(cudaMemcpyAsync(I.gr.p, r0, vb, cudaMemcpyDeviceToDevice, c->st));
  std::vector<double> rn(nrhs), rn0(nrhs);
  std::vector<char> done(nrhs, 0);
  for (int r = 0; r < nrhs; ++r) {
    double n2;
    OV_TRY(norm2(c, I.pv, I.gr.c() + r * v1, V, &n2));
    rn[r] = rn0[r] = std::sqrt(n2);
    done[r] = !(rn0[r] > 0.0);
  }
  const bool is16 = (I.p == OP_F16 || I.p == OP_B16);
  int n_inner = 0, k = 0, step = 0;
  while (n_inner < maxit) {
    bool all = true;
    for (int r = 0; r < nrhs; ++r) all = all && done[r];
    if (all) break;
    if (k == dirs) k = 0;  // restart: drop the kept directions
    char* u = I.gu.c() + (size_t)k * vb;
    char* cd = I.gc.c() + (size_t)k * vb;
    // inner right-hand sides r / |r| (zero for finished RHS)
    for (int r = 0; r < nrhs; ++r) {
      launch_axpby(I.pv, done[r] ? 0.0 : 1.0 / rn[r], I.gr.c() + r * v1, 0.0, nullptr, I.grhs.c() + r * v1, V, 1,
                   c->st);
      OV_TRY(launched(c));
    }
    int its = 0;
    double est = 0.0;
    OV_TRY(sumr_core(c, S, c->coef_relaxed, mu, I.grhs.p, u, nrhs, c->gm_tol, std::min(c->gm_maxit, maxit - n_inner),
                     &its, &est));
    n_inner += its;
    // c_k = D[mu] u_k with the accurate order
    double umax = 0.0;
    std::vector<double> un(nrhs, 0.0);
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      double n2;
      OV_TRY(norm2(c, I.pv, u + r * v1, V, &n2));
      un[r] = std::sqrt(n2);
      umax = std::max(umax, un[r]);
    }
    if (!(umax > 0.0) || !std::isfinite(umax)) return fail(c, OV_ERR_NOT_CONVERGED, "GCR: inner solve returned zero");
    const double scale = is16 ? std::sqrt(24.0 * (double)V) / umax : 1.0;
    OV_TRY(sign_core(c, I, u, cd, nrhs, K_OVL, mu, scale));
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      const size_t o = r * v1;
      for (int i = 0; i < k; ++i) {  // modified Gram-Schmidt against the kept c_i
        const char* ci = I.gc.c() + (size_t)i * vb + o;
        const char* ui = I.gu.c() + (size_t)i * vb + o;
        double2 be;
        OV_TRY(dots(c, I.pv, ci, cd + o, V, &be));
        launch_caxpy(I.pv, make_double2(-be.x, -be.y), ci, cd + o, V, 1, c->st);
        launch_caxpy(I.pv, make_double2(-be.x, -be.y), ui, u + o, V, 1, c->st);
        OV_TRY(launched(c, 2));
      }
      double n2;
      OV_TRY(norm2(c, I.pv, cd + o, V, &n2));
      const double nc = std::sqrt(n2);
      if (!(nc > 0.0) || !std::isfinite(nc)) return fail(c, OV_ERR_NOT_CONVERGED, "GCR: direction not finite or zero");
      launch_axpby(I.pv, 1.0 / nc, cd + o, 0.0, nullptr, cd + o, V, 1, c->st);
      launch_axpby(I.pv, 1.0 / nc, u + o, 0.0, nullptr, u + o, V, 1, c->st);
      OV_TRY(launched(c, 2));
      double2 g;
      OV_TRY(dots(c, I.pv, cd + o, I.gr.c() + o, V, &g));
      launch_caxpy(I.pv, g, u + o, static_cast<char*>(e) + o, V, 1, c->st);
      launch_caxpy(I.pv, make_double2(-g.x, -g.y), cd + o, I.gr.c() + o, V, 1, c->st);
      OV_TRY(launched(c, 2));
      OV_TRY(norm2(c, I.pv, I.gr.c() + o, V, &n2));
      rn[r] = std::sqrt(n2);
      if (!std::isfinite(rn[r])) return fail(c, OV_ERR_NOT_CONVERGED, "GCR residual not finite");
      if (rn[r] <= tol * rn0[r]) done[r] = 1;
    }
    ++k;
    ++step;
  }
  *inner = n_inner;
  *steps = step;
  for (int r = 0; r < nrhs; ++r)
    if (!done[r]) return OV_ERR_NOT_CONVERGED;  // caller decides
  return OV_OK;
}

// Builds the FP32 operator instance (c->mid) from device links in the
// interface layout; a failure leaves the context without it.
ov_status build_fp32_operator(ov_ctx* c, const void* dl) {
  ov_status s = init_inst(c, c->mid, OP_F32, dl);
  if (s == OV_OK && c->configured && c->n_ev > 0) {  // eigenvectors from the FP64 copy
    cudaError_t e = c->mid.evecs.ensure(c->mid.vbytes(c->g.V) * c->n_ev);
    if (e != cudaSuccess) {
      s = fail(c, e == cudaErrorMemoryAllocation ? OV_ERR_NOMEM : OV_ERR_CUDA, cudaGetErrorString(e));
    } else {
      launch_convert(OP_F64, OP_F32, c->hi.evecs.p, c->mid.evecs.p, c->g.V, c->n_ev, 1.0, 0, c->st);
      s = launched(c);
    }
  }
  if (s == OV_OK) {
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) s = fail(c, OV_ERR_CUDA, cudaGetErrorString(e));
  }
  if (s != OV_OK) {
    c->mid.release();
    c->mid.active = false;
  }
  return s;
}

// The FP32 GCR level for a 16-bit context, from the context's own FP64 links.
ov_status ensure_fp32_level(ov_ctx* c) {
  if (!c->gm_fp32 || c->mid.active || (c->prec != OV_MIXED_FP16 && c->prec != OV_MIXED_BF16)) return OV_OK;
  DevBuf iface;
  OV_CK(iface.ensure((size_t)c->g.V * 4 * 9 * 16));
  launch_unpack_links_f64(c->g, c->hi.links.p, iface.p, c->st);
  OV_TRY(launched(c));
  const ov_status s = build_fp32_operator(c, iface.p);
  iface.release();
  return s;
}

static ov_status gmresr_core(ov_ctx* c, double mu, double tol, int maxit, const void* b, void* x, int nrhs,
                             ov_dtype dt, int* iters, double* true_rel_resid) {
  if (!c) return OV_ERR_INVALID;
  if (!b || !x) return fail(c, OV_ERR_INVALID, "null vector");
  if (!std::isfinite(mu) || !(std::fabs(mu) < 1.0) || !(tol > 0.0) || maxit < 1)
    return fail(c, OV_ERR_INVALID, "need |mu| < 1, tol > 0, maxit >= 1");
  OV_TRY(check_dtype(c, nrhs, dt));
  if (!c->configured) return fail(c, OV_ERR_STATE, "sign(K) not configured: call ov_sign_config first");
  OV_TRY(relaxed_coefficients(c));
  OV_TRY(ensure_fp32_level(c));
  c->stats.gmresr_order = (int)c->coef_relaxed.size() - 1;
  c->stats.inner_iterations = 0;
  c->stats.outer_iterations = 0;
  c->res_history.clear();
  c->stats.gcr_iterations = 0;
  Inst& H = c->hi;
  // S: the inner SUMR level (the context precision); I: the GCR level, the
  // FP32 operator (built on first use, or by ov_enable_fp32_operator) when a
  // 16-bit context has one
  Inst& S = (c->prec == OV_FP64) ? c->hi : c->lo;
  const bool mid = c->mid.active && (c->prec == OV_MIXED_FP16 || c->prec == OV_MIXED_BF16);
  Inst& I = mid ? c->mid : S;
  const int64_t V = c->g.V;
  const size_t v1 = H.vbytes(V), vb = v1 * nrhs, iv1 = I.vbytes(V);
  OV_TRY(ensure_work(c, H, nrhs));
  OV_TRY(ensure_work(c, I, nrhs));
  OV_TRY(ensure_work(c, S, nrhs));
  OV_CK(c->o_x.ensure(vb));
  OV_CK(c->o_r.ensure(vb));
  OV_CK(c->o_rhs.ensure(vb));
  OV_CK(c->o_q.ensure(vb));
  OV_CK(I.cx.ensure(iv1 * nrhs));
  OV_TRY(pack_input(c, H, b, nrhs, dt, c->o_rhs.p));
  std::vector<double> rhs_n(nrhs), res(nrhs), rn(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    double n2;
    OV_TRY(norm2(c, OP_F64, c->o_rhs.c() + r * v1, V, &n2));
    rhs_n[r] = std::sqrt(n2);
    res[r] = rhs_n[r] > 0 ? 1.0 : 0.0;
    rn[r] = rhs_n[r];
  }
  OV_CK(cudaMemsetAsync(c->o_x.p, 0, vb, c->st));
  OV_CK(cudaMemcpyAsync(c->o_r.p, c->o_rhs.p, vb, cudaMemcpyDeviceToDevice, c->st));
  // Defect correction as in the CG solver, on D[mu] itself: r = b - D x
  // (FP64), GCR on D e = r / |r| in the context precision, x += |r| e.
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
    int its = 0, steps = 0;
    ov_status s = gcr_core(c, I, S, I.xin.p, I.cx.p, nrhs, mu, inner, maxit - total, &its, &steps);
    total += its;
    c->stats.gcr_iterations += steps;
    if (s != OV_OK && s != OV_ERR_NOT_CONVERGED) return s;
    for (int r = 0; r < nrhs; ++r) {
      launch_convert(I.pv, OP_F64, I.cx.c() + r * iv1, c->o_x.c() + r * v1, V, 1, rn[r], 1, c->st);
      OV_TRY(launched(c));
    }
    c->stats.outer_iterations++;
    OV_TRY(sign_core(c, H, c->o_x.p, c->o_q.p, nrhs, K_OVL, mu, 1.0));
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
  if (!ok) return fail(c, OV_ERR_NOT_CONVERGED, "GMRESR stopped before reaching tol");
  return OV_OK;
}

}  // namespace ov

extern "C" {


ov_status ov_enable_fp32_operator(ov_ctx* c, const void* links) {
  if (!c) return OV_ERR_INVALID;
  if (!links) return fail(c, OV_ERR_INVALID, "null links");
  if (c->prec != OV_MIXED_FP16 && c->prec != OV_MIXED_BF16) return OV_OK;  // already FP32 or FP64
  if (c->mid.active) return OV_OK;
  const void* dl = nullptr;
  ov_status s = stage_in(c, c->stage_links, links, (size_t)c->g.V * 4 * 9 * 16, &dl);
  if (s == OV_OK) s = build_fp32_operator(c, dl);
  c->stage_links.release();
  return s;
}

ov_status ov_set_gmresr_fp32_level(ov_ctx* c, int on) {
  if (!c) return OV_ERR_INVALID;
  c->gm_fp32 = on != 0;
  if (!c->gm_fp32 && c->mid.active) {  // back to GCR in the storage precision
    OV_CK(cudaStreamSynchronize(c->st));
    c->mid.release();
    c->mid.active = false;
  }
  return OV_OK;
}

ov_status ov_set_gmresr_params(ov_ctx* c, int inner_order, double inner_tol, int inner_maxit, int max_dirs) {
  if (!c) return OV_ERR_INVALID;
  if (inner_order < 0 || !(inner_tol > 0.0 && inner_tol < 1.0) || inner_maxit < 1 || max_dirs < 1 || max_dirs > 64)
    return fail(c, OV_ERR_INVALID, "need inner_order >= 0, 0 < inner_tol < 1, inner_maxit >= 1, 1 <= max_dirs <= 64");
  c->gm_order = inner_order;
  c->gm_tol = inner_tol;
  c->gm_maxit = inner_maxit;
  c->gm_dirs = max_dirs;
  c->coef_relaxed.clear();
  return OV_OK;
}

ov_status ov_sumr(ov_ctx* c, double mu, double tol, int maxit, const void* b, void* x, int nrhs, ov_dtype dt,
                  int* iters, double* est_rel_resid) {
  if (!c) return OV_ERR_INVALID;
  if (!b || !x) return fail(c, OV_ERR_INVALID, "null vector");
  if (!std::isfinite(mu) || !(std::fabs(mu) < 1.0) || !(tol >= 0.0) || maxit < 0)
    return fail(c, OV_ERR_INVALID, "need |mu| < 1, tol >= 0, maxit >= 0");
  OV_TRY(check_dtype(c, nrhs, dt));
  if (!c->configured) return fail(c, OV_ERR_STATE, "sign(K) not configured: call ov_sign_config first");
  Inst& I = c->op();
  OV_TRY(ensure_work(c, I, nrhs));
  OV_CK(I.cx.ensure(I.vbytes(c->g.V) * nrhs));
  OV_TRY(pack_input(c, I, b, nrhs, dt, I.xin.p));
  int it = 0;
  double est = 0.0;
  OV_TRY(sumr_core(c, I, c->coef, mu, I.xin.p, I.cx.p, nrhs, tol, maxit, &it, &est));
  c->stats.inner_iterations = it;
  OV_TRY(unpack_output(c, I, I.cx.p, x, nrhs, dt));
  if (iters) *iters = it;
  if (est_rel_resid) *est_rel_resid = est;
  return OV_OK;
}

ov_status ov_solve_gmresr(ov_ctx* c, double mu, double tol, int maxit, const void* b, void* x, int nrhs,
                          ov_dtype dt, int* iters, double* true_rel_resid) {
  return gmresr_core(c, mu, tol, maxit, b, x, nrhs, dt, iters, true_rel_resid);
}

}  // extern "C"
