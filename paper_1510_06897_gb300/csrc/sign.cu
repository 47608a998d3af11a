// The sign(K) driver (Eq. 3) and the overlap operators built on it (Eq. 1):
// Chebyshev coefficients on the host, the deflation projection, the Clenshaw
// recurrence as 2N stencil launches with the polynomial algebra in their
// epilogues, and the final launch that assembles sign(K), D[mu], D[mu]^dagger
// or the chiral-sector operator.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace ov {

// Chebyshev-Gauss interpolation of y^{-1/2} on [a^2, b^2] (Eq. 3 reading):
// c_j = 2/(N+1) sum_k f(y_k) cos(j theta_k), theta_k = pi (k + 1/2)/(N + 1).
std::vector<double> chebyshev_coefficients(int order, double a, double b) {
  const int n1 = order + 1;
  std::vector<double> f(n1), c(n1);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n1; ++k) {
    const double th = pi * (k + 0.5) / n1;
    const double y = 0.5 * ((b * b - a * a) * std::cos(th) + b * b + a * a);
    f[k] = 1.0 / std::sqrt(y);
  }
  for (int j = 0; j < n1; ++j) {
    double s = 0.0;
    for (int k = 0; k < n1; ++k) s += f[k] * std::cos(j * pi * (k + 0.5) / n1);
    c[j] = 2.0 * s / n1;
  }
  return c;
}

// K applied to a recurrence vector: out (storage I.p) = s1 K in + sum w_j v_j.
ov_status k_step(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, const EpiArgs& e) {
  return dslash(c, I, I.p, in, out, e, nrhs);
}

// sign(K) / D[mu] / D[mu]^dagger on nrhs vectors in I.pv storage.
// scale: the recurrence runs on scale * (input); results are unscaled in the
// final epilogue (used to keep 16-bit storage in range).
// max over [a^2, b^2] of |sqrt(y) f_N(y) - 1|, f_N = c_0/2 + sum_j c_j T_j(z),
// sampled at 2049 Chebyshev-Lobatto points of z (dense near both ends).
double chebyshev_sign_error(const std::vector<double>& cf, double a, double b) {
  const int n = (int)cf.size() - 1, M = 2049;
  const double pi = 3.14159265358979323846;
  double worst = 0.0;
  for (int i = 0; i < M; ++i) {
    const double z = std::cos(pi * i / (M - 1));
    const double y = 0.5 * ((b * b - a * a) * z + b * b + a * a);
    double b1 = 0.0, b2 = 0.0;  // Clenshaw for sum_{j>=1} c_j T_j(z) + c_0/2
    for (int j = n; j >= 1; --j) {
      const double b0 = 2.0 * z * b1 - b2 + cf[j];
      b2 = b1;
      b1 = b0;
    }
    const double f = z * b1 - b2 + 0.5 * cf[0];
    worst = std::max(worst, std::fabs(std::sqrt(y) * f - 1.0));
  }
  return worst;
}

ov_status sign_core(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, Kind kind, double mu, double scale,
                    const std::vector<double>* cf_override) {
  if (!c->configured) return fail(c, OV_ERR_STATE, "sign(K) not configured: call ov_sign_config first");
  OV_TRY(ensure_work(c, I, nrhs));
  const int64_t V = c->g.V;
  const size_t vb = I.vbytes(V), pb = I.pbytes(V);
  const int g5in = (kind == K_OVL_DAG);
  const int n_ev = c->n_ev;

  // S3: deflation projection c_i = phi_i^dagger psi, psi_perp = psi - sum c_i phi_i,
  //     d = sum sgn(lambda_i) c_i phi_i  (both scaled by `scale`).  Several
  //     right-hand sides: one Gram launch reads every eigenvector once for all
  //     of them (c stored [i][r]); one right-hand side: the projection kernel.
  //     The tensor-core Gram takes up to 128 eigenvectors, the CUDA-core one 64.
  const char* mode = std::getenv("OV_DEFL_GEMM");
  const bool tc = I.pv == OP_F32 && n_ev > 0 && nrhs > 1 && n_ev <= tc_gram_max_rows() &&
                  nrhs <= tc_gram_max_rhs() && !(mode && std::strcmp(mode, "cuda") == 0);
  const bool batched = n_ev > 0 && nrhs > 1 && (tc || (n_ev <= gram_max_vectors() && nrhs <= gram_max_vectors()));
  if (batched) {
    OV_CK(c->d_gram.ensure(sizeof(double2) * (size_t)n_ev * nrhs * kReduceBlocks));
    int nblk = kReduceBlocks;
    if (tc) {
      // tensor cores: one CTA per SM, TF32 x 3 split products
      nblk = std::min(c->num_sms, kReduceBlocks);
      OV_CK(c->d_err.ensure(sizeof(int)));
      OV_CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(int), c->st));
      OV_CK(launch_tc_gram(I.evecs.p, n_ev, in, nrhs, V, g5in, c->d_gram.as<double2>(), nblk, c->d_err.as<int>(),
                           c->stall_cycles > 0 ? c->d_never.as<int>() : nullptr, c->stall_cycles, c->st));
      OV_TRY(launched(c));
      c->stats.tc_gemm_launches++;
      int herr = 0;
      OV_CK(cudaMemcpyAsync(&herr, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      OV_CK(cudaStreamSynchronize(c->st));
      if (herr) return fail(c, OV_ERR_CUDA, "tensor-core projection: a bounded wait expired");
    } else {
      OV_CK(launch_gram(I.pv, I.evecs.p, n_ev, in, nrhs, V, c->d_gram.as<double2>(), kReduceBlocks, c->st, g5in));
      OV_TRY(launched(c));
    }
    launch_reduce_partials(c->d_gram.as<double2>(), n_ev * nrhs, nblk, c->d_c.as<double2>(), c->st);
    OV_TRY(launched(c));
  }
  if (batched && I.pv == OP_F32 && n_ev <= 128) {
    launch_defl_combine_multi(I.p, c->g, I.evecs.p, n_ev, c->d_c.as<double2>(), nrhs, c->d_sgn.as<double>(), in,
                              g5in, scale, I.perp.p, I.d.p, c->st);
    OV_TRY(launched(c));
  } else {
    for (int r = 0; r < nrhs; ++r) {
      const char* in_r = static_cast<const char*>(in) + r * vb;
      double2* cr = batched ? c->d_c.as<double2>() + r : c->d_c.as<double2>() + (size_t)r * std::max(1, n_ev);
      const int cstride = batched ? nrhs : 1;
      if (n_ev > 0 && !batched) {
        launch_defl_dot(I.pv, c->g, I.evecs.p, n_ev, in_r, g5in, c->d_partial.as<double2>(), c->st);
        OV_TRY(launched(c));
        launch_reduce_partials(c->d_partial.as<double2>(), n_ev, kReduceBlocks, cr, c->st);
        OV_TRY(launched(c));
      }
      launch_defl_combine(I.pv, I.p, c->g, I.evecs.p, n_ev, cr, cstride, c->d_sgn.as<double>(), in_r, g5in, scale,
                          I.perp.c() + r * pb, n_ev > 0 ? I.d.c() + r * vb : nullptr, c->st);
      OV_TRY(launched(c));
    }
  }

  // S4: backward (Clenshaw) recurrence for f_N(Z) psi_perp, Z = alpha K^2 + beta:
  //   b_k = c_k psi_perp + 2 Z b_{k+1} - b_{k+2},  k = N-1 .. 1,  b_N = c_N psi_perp,
  //   h   = (b_0 - b_2)/2 = c_0/2 psi_perp + Z b_1 - b_2.
  // Each Z application is two stencil launches; the second carries the
  // recurrence algebra in its epilogue.
  const double a2 = c->a * c->a, b2 = c->b * c->b;
  const double alpha = 2.0 / (b2 - a2), beta = -(b2 + a2) / (b2 - a2);
  const std::vector<double>& cf = cf_override ? *cf_override : c->coef;
  const int N = (int)cf.size() - 1;
  void* perp = I.perp.p;
  struct Vec {
    void* p;
    double s;
  };
  Vec b1{perp, cf[N]}, b2v{nullptr, 0.0};
  void* h = nullptr;
  if (c->prof == 2) OV_TRY(prof_open(c));
  for (int k = N - 1; k >= 0; --k) {
    EpiArgs ek;
    ek.m_w = c->m_w;
    OV_TRY(k_step(c, I, b1.p, I.t.p, nrhs, ek));  // t = K b1.p
    void* dst = (b2v.p != nullptr && b2v.p != perp) ? b2v.p : (b1.p == I.bA.p ? I.bB.p : I.bA.p);
    EpiArgs e;
    e.m_w = c->m_w;
    const double zs = (k > 0) ? 2.0 : 1.0;  // last step builds (b_0 - b_2)/2
    e.s1 = zs * alpha * b1.s;
    e.v[0] = b1.p;
    e.w[0] = zs * beta * b1.s;
    e.v[1] = b2v.p;
    e.w[1] = -b2v.s;
    e.v[2] = perp;
    e.w[2] = (k > 0) ? cf[k] : 0.5 * cf[0];
    OV_TRY(k_step(c, I, I.t.p, dst, nrhs, e));
    b2v = b1;
    b1 = Vec{dst, 1.0};
    h = dst;
  }
  if (c->prof == 2) OV_TRY(prof_close(c, 2 * N));

  // S5: out = K h (= P(K) psi_perp) + d, with the overlap assembly (Eq. 1) fused:
  //   sign:   out = (K h + d) / scale
  //   D:      out = (1+mu)/2 in + (1-mu)/2 gamma5 (K h + d) / scale
  //   D^dag:  out = (1+mu)/2 in + (1-mu)/2 (K h + d) / scale     (input was gamma5 in)
  //   chiral: out = c0 in + c1 P (K h + d) / scale, c0 = [(1+mu)^2 + (1-mu)^2]/4,
  //           c1 = +-(1 - mu^2)/2, P the projector on the input's chirality
  EpiArgs e;
  e.m_w = c->m_w;
  const bool chiral = (kind == K_CHI_P || kind == K_CHI_M);
  const double c1 = 0.5 * (1.0 - mu * mu) * (kind == K_CHI_P ? 1.0 : -1.0);
  const double f = (kind == K_SIGN ? 1.0 : chiral ? c1 : 0.5 * (1.0 - mu)) / scale;
  e.s1 = f;
  e.z = n_ev > 0 ? I.d.p : nullptr;
  e.wz = f;
  e.g5_out = (kind == K_OVL);
  if (kind != K_SIGN) {
    e.y = in;
    e.c0 = chiral ? 0.25 * ((1.0 + mu) * (1.0 + mu) + (1.0 - mu) * (1.0 - mu)) : 0.5 * (1.0 + mu);
  }
  if (chiral) e.keep_half = (kind == K_CHI_P) ? 0 : 1;
  OV_TRY(dslash(c, I, I.pv, h, out, e, nrhs));
  c->stats.sign_applies += nrhs;
  return OV_OK;
}

// out = D^dagger D in (vectors in I.pv), through I.tmp.
ov_status normal_apply(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, double mu, double scale) {
  OV_TRY(ensure_work(c, I, nrhs));
  OV_TRY(sign_core(c, I, in, I.tmp.p, nrhs, K_OVL, mu, scale));
  return sign_core(c, I, I.tmp.p, out, nrhs, K_OVL_DAG, mu, scale);
}

ov_status op_apply(ov_ctx* c, Inst& I, const void* in, void* out, int nrhs, double mu, double scale, int chirality) {
  if (chirality == 0) return normal_apply(c, I, in, out, nrhs, mu, scale);
  return sign_core(c, I, in, out, nrhs, chirality > 0 ? K_CHI_P : K_CHI_M, mu, scale);
}

}  // namespace ov
