// ov_eigs: the lowest-|lambda| eigenpairs of K that the deflation of Eq. 3
// needs (Sec. 2 precomputes them with a polynomial-preconditioned implicitly
// restarted Lanczos).  Here: block subspace iteration on K^2 with a scaled
// Chebyshev filter that damps [cut^2, b^2] (cut = largest Ritz value of the
// block), Rayleigh-Ritz with K^2 (which orders the block and sets the filter
// bounds), then Rayleigh-Ritz with K inside the lowest K^2 cluster so that
// +lambda and -lambda split.
// All inner products are FP64 sums; the m x m Hermitian eigenproblems are
// solved on the host by cyclic Jacobi rotations.
#include <algorithm>
#include <complex>
#include <cstdlib>

#include "ctx.h"

using namespace ov;
using cd = std::complex<double>;

namespace {

// Eigen-decomposition of a Hermitian n x n matrix A (row-major, overwritten):
// ascending eigenvalues w, eigenvectors as the columns of V (row-major).
// Householder reflections reduce A to a tridiagonal matrix whose complex
// off-diagonal entries a diagonal phase transform makes real; the implicit
// QL iteration with Wilkinson-type shifts diagonalises that real symmetric
// tridiagonal matrix, accumulating its rotations; V = Q diag(phase) Z.
// O(n^3) once instead of per sweep of cyclic Jacobi (25x faster at n = 102).
void herm_eig(int n, std::vector<cd>& A, std::vector<double>& w, std::vector<cd>& V) {
  auto a = [&](int i, int j) -> cd& { return A[(size_t)i * n + j]; };
  // Q: accumulated reflections (row-major), starts as the identity
  std::vector<cd> Q((size_t)n * n, cd(0.0));
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<cd> v(n), p(n), wv(n);
  for (int k = 0; k + 2 < n; ++k) {
    // reflect x = A[k+1.., k] onto alpha e_1
    double xn2 = 0.0;
    for (int i = k + 1; i < n; ++i) xn2 += std::norm(a(i, k));
    const double xn = std::sqrt(xn2);
    if (xn == 0.0) continue;
    const cd x0 = a(k + 1, k);
    const cd ph = (std::abs(x0) > 0.0) ? x0 / std::abs(x0) : cd(1.0);
    const cd alpha = -ph * xn;
    for (int i = k + 1; i < n; ++i) v[i] = a(i, k);
    v[k + 1] -= alpha;
    double vn2 = 0.0;
    for (int i = k + 1; i < n; ++i) vn2 += std::norm(v[i]);
    if (vn2 == 0.0) continue;
    const double vn = std::sqrt(vn2);
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    // H = I - 2 v v^dagger on rows / columns k+1..n-1:  A <- H A H
    // p = 2 A_sub v ; K = v^dagger p (real) ; w = p - K v ; A_sub <- A_sub - v w^dagger - w v^dagger
    for (int i = k + 1; i < n; ++i) {
      cd s = 0.0;
      for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
      p[i] = 2.0 * s;
    }
    cd K = 0.0;
    for (int i = k + 1; i < n; ++i) K += std::conj(v[i]) * p[i];
    for (int i = k + 1; i < n; ++i) wv[i] = p[i] - K * v[i];
    for (int i = k + 1; i < n; ++i)
      for (int j = k + 1; j < n; ++j) a(i, j) -= v[i] * std::conj(wv[j]) + wv[i] * std::conj(v[j]);
    a(k + 1, k) = alpha;
    a(k, k + 1) = std::conj(alpha);
    for (int i = k + 2; i < n; ++i) a(i, k) = a(k, i) = 0.0;
    // Q <- Q H (columns k+1..n-1)
    for (int r = 0; r < n; ++r) {
      cd s = 0.0;
      for (int j = k + 1; j < n; ++j) s += Q[(size_t)r * n + j] * v[j];
      s *= 2.0;
      for (int j = k + 1; j < n; ++j) Q[(size_t)r * n + j] -= s * std::conj(v[j]);
    }
  }
  // T = Q^dagger A Q: real diagonal d, complex subdiagonal; phases make it real
  std::vector<double> d(n), e(n, 0.0);
  std::vector<cd> phase(n, cd(1.0));
  for (int i = 0; i < n; ++i) d[i] = a(i, i).real();
  for (int i = 0; i + 1 < n; ++i) {
    const cd s = a(i + 1, i);
    const double m = std::abs(s);
    e[i] = m;
    phase[i + 1] = (m > 0.0) ? phase[i] * (s / m) : phase[i];
  }
  // implicit QL on (d, e), rotations accumulated into Z (row-major, real)
  std::vector<double> Z((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 60; ++iter) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-16 * dd) break;
      }
      if (m == l) break;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = m - 1;
      for (; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pp;
          e[m] = 0.0;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        for (int k = 0; k < n; ++k) {
          const double z1 = Z[(size_t)k * n + i + 1], z0 = Z[(size_t)k * n + i];
          Z[(size_t)k * n + i + 1] = s * z0 + c * z1;
          Z[(size_t)k * n + i] = c * z0 - s * z1;
        }
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  // ascending order; V = Q diag(phase) Z
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] != d[y] ? d[x] < d[y] : x < y; });
  w.resize(n);
  V.assign((size_t)n * n, cd(0.0));
  for (int jj = 0; jj < n; ++jj) {
    const int j = ord[jj];
    w[jj] = d[j];
    for (int r = 0; r < n; ++r) {
      cd s = 0.0;
      for (int k = 0; k < n; ++k) s += Q[(size_t)r * n + k] * phase[k] * Z[(size_t)k * n + j];
      V[(size_t)r * n + jj] = s;
    }
  }
}

// Generalised Rayleigh-Ritz: eigenpairs of H in the metric G (both m x m
// Hermitian): G = V g V^dag, S = V g^{-1/2}, S^dag H S = Q diag(w) Q^dag,
// returns w ascending and C = S Q (row-major, columns = Ritz coefficients).
void rayleigh_ritz(int m, const std::vector<cd>& G, const std::vector<cd>& H, std::vector<double>& w,
                   std::vector<cd>& C) {
  std::vector<cd> Gc = G;
  std::vector<double> gw;
  std::vector<cd> gv;
  herm_eig(m, Gc, gw, gv);
  double gmax = 0;
  for (double x : gw) gmax = std::max(gmax, x);
  std::vector<cd> S((size_t)m * m), T1((size_t)m * m, 0.0), Hp((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) S[(size_t)i * m + j] = gv[(size_t)i * m + j] / std::sqrt(std::max(gw[j], 1e-14 * gmax));
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k) {
      const cd h = 0.5 * (H[(size_t)i * m + k] + std::conj(H[(size_t)k * m + i]));
      for (int j = 0; j < m; ++j) T1[(size_t)i * m + j] += h * S[(size_t)k * m + j];
    }
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k) {
      const cd s = std::conj(S[(size_t)k * m + i]);
      for (int j = 0; j < m; ++j) Hp[(size_t)i * m + j] += s * T1[(size_t)k * m + j];
    }
  std::vector<double> th;
  std::vector<cd> q;
  herm_eig(m, Hp, th, q);
  std::vector<int> ord(m);
  for (int i = 0; i < m; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return th[x] != th[y] ? th[x] < th[y] : x < y; });
  w.resize(m);
  C.assign((size_t)m * m, 0.0);
  for (int jj = 0; jj < m; ++jj) {
    w[jj] = th[ord[jj]];
    for (int i = 0; i < m; ++i) {
      cd acc = 0.0;
      for (int k = 0; k < m; ++k) acc += S[(size_t)i * m + k] * q[(size_t)k * m + ord[jj]];
      C[(size_t)i * m + jj] = acc;
    }
  }
}

// out[i * mb + j] = <A_i, B_j> (FP64 sums), in tiles of at most
// gram_max_vectors() vectors per side (one Gram launch per tile).
ov_status gram(ov_ctx* c, OpPrec p, const void* A, int ma, const void* B, int mb, DevBuf& partial,
               std::vector<cd>& out) {
  const int64_t V = c->g.V;
  const size_t vb = (size_t)spinor_bytes_per_site(p) * V;
  const int tile = gram_max_vectors();
  out.assign((size_t)ma * mb, cd(0.0));
  OV_CK(partial.ensure(sizeof(double2) * (size_t)tile * tile * kReduceBlocks));
  std::vector<double2> r((size_t)tile * tile);
  for (int i0 = 0; i0 < ma; i0 += tile)
    for (int j0 = 0; j0 < mb; j0 += tile) {
      const int ni = std::min(tile, ma - i0), nj = std::min(tile, mb - j0);
      OV_CK(launch_gram(p, static_cast<const char*>(A) + (size_t)i0 * vb, ni,
                        static_cast<const char*>(B) + (size_t)j0 * vb, nj, V, partial.as<double2>(), kReduceBlocks,
                        c->st));
      OV_TRY(launched(c));
      OV_TRY(read_reduced(c, partial.as<double2>(), ni * nj, r.data()));
      for (int i = 0; i < ni; ++i)
        for (int j = 0; j < nj; ++j) {
          const double2 v = r[(size_t)i * nj + j];
          out[(size_t)(i0 + i) * mb + j0 + j] = cd(v.x, v.y);
        }
    }
  return OV_OK;
}

// Largest block of the subspace iteration (vectors); the Gram matrices are
// formed in tiles, the stencil and the rotation take any width.
constexpr int kEigsMaxBlock = 128;

}  // namespace

extern "C" ov_status ov_eigs(ov_ctx* c, int n_ev, double tol, int max_iter, double* evals, void* evecs,
                             double* lambda_max_out) {
  if (!c) return OV_ERR_INVALID;
  if (!evals || !evecs) return fail(c, OV_ERR_INVALID, "null output");
  const int mmax = kEigsMaxBlock;
  if (n_ev < 1 || n_ev + 8 > mmax) return fail(c, OV_ERR_INVALID, "need 1 <= n_ev <= " + std::to_string(mmax - 8));
  if (!(tol > 0.0) || max_iter < 1) return fail(c, OV_ERR_INVALID, "need tol > 0 and max_iter >= 1");
  const int64_t V = c->g.V;
  // block of ~2.5 n_ev (at most kEigsMaxBlock): a wider block separates the
  // wanted band from the rest better, so fewer filter sweeps are needed
  // (counted on a model problem: 20 pairs, block 50 vs 30, half the K
  // applications)
  const int m = std::min(mmax, std::max(n_ev + 8, (5 * n_ev) / 2));
  if ((int64_t)m > 12 * V) return fail(c, OV_ERR_INVALID, "block larger than the vector space");
  Inst& I = (c->prec == OV_FP32) ? c->lo : c->hi;  // FP32 or FP64 storage (I.p == I.pv)
  const OpPrec P = I.p;
  const size_t vb = I.vbytes(V);
  DevBuf bA, bB, bT, partial, dq;
  OV_CK(bA.ensure(vb * m));
  OV_CK(bB.ensure(vb * m));
  OV_CK(bT.ensure(vb * m));
  OV_TRY(ensure_work(c, I, 1));

  launch_random_block(P, bA.p, m, V, 0x0ddc0ffeeull, c->st);
  OV_TRY(launched(c));

  // |lambda|_max: power iteration on K^2, then a safety margin; never below 6.5,
  // which the free field attains.
  double lam_est = 0.0;
  {
    double n0;
    OV_TRY(norm2(c, P, bA.p, V, &n0));
    launch_axpby(P, 1.0 / std::sqrt(n0), bA.p, 0.0, nullptr, bB.p, V, 1, c->st);
    OV_TRY(launched(c));
    for (int it = 0; it < 30; ++it) {
      EpiArgs e;
      e.m_w = c->m_w;
      OV_TRY(k_step(c, I, bB.p, bT.p, 1, e));
      OV_TRY(k_step(c, I, bT.p, I.tmp.p, 1, e));
      double2 rq;
      OV_TRY(dots(c, P, bB.p, I.tmp.p, V, &rq));
      lam_est = std::sqrt(std::max(rq.x, 0.0));
      double nn;
      OV_TRY(norm2(c, P, I.tmp.p, V, &nn));
      launch_axpby(P, 1.0 / std::sqrt(nn), I.tmp.p, 0.0, nullptr, bB.p, V, 1, c->st);
      OV_TRY(launched(c));
    }
  }
  const double bmax = std::max(6.5, 1.02 * lam_est);
  const double b2 = bmax * bmax;

  std::vector<double> theta(m, 0.0), res(m, 1.0);
  double cut2 = b2 * 0.5, low2 = 0.0;
  void* Y = bA.p;  // current block
  void* Z = bB.p;  // scratch block
  bool converged = false;
  int iter = 0;
  // Filter degree per iteration: as high as possible (fewer Rayleigh-Ritz
  // steps; on the dense low band of the 24^3 x 48 field, 41 pairs: 21 steps at
  // degree 32, 10 at 64, 7 at 96, about the same number of stencil
  // applications in total), but no higher than keeps the filter's ratio
  // between the block's lowest Ritz value and its top (the damped interval's
  // edge) within kFilterRange: a larger spread leaves the block's upper
  // vectors below the precision of its Gram matrix, and the pairs near the
  // top of the wanted band stop converging (seen on a 4^4 lattice, 30 pairs,
  // degree 96).  OV_EIGS_DEGREE (4 .. 256) overrides the upper limit of 96.
  int degree = 96;
  constexpr double kFilterRange = 1e4;
  if (const char* env = std::getenv("OV_EIGS_DEGREE")) degree = std::min(256, std::max(4, std::atoi(env)));
  for (; iter < max_iter; ++iter) {
    if (iter > 0) {
      // scaled Chebyshev filter on K^2 damping [cut2, b2], normalised at 0 (a
      // lower bound of the spectrum of K^2): every component is scaled by at
      // most 1, so no filter degree can overflow the block's storage
      const double e = 0.5 * (b2 - cut2), cc = 0.5 * (b2 + cut2);
      const double x_low = std::fabs((low2 - cc) / e);  // > 1: the block's lowest Ritz value
      const int deg_iter = std::max(
          std::min(4, degree),
          std::min(degree, (int)(std::acosh(kFilterRange) / std::acosh(std::max(x_low, 1.0 + 1e-12)))));
      double sigma = e / (0.0 - cc);
      const double sigma1 = sigma, gam = 2.0 / sigma1;
      EpiArgs ek;
      ek.m_w = c->m_w;
      OV_TRY(k_step(c, I, Y, bT.p, m, ek));
      EpiArgs e1;
      e1.m_w = c->m_w;
      e1.s1 = sigma / e;
      e1.v[0] = Y;
      e1.w[0] = -sigma * cc / e;
      OV_TRY(k_step(c, I, bT.p, Z, m, e1));
      void* y0 = Y;
      void* y1 = Z;
      for (int k = 2; k <= deg_iter; ++k) {
        const double sn = 1.0 / (gam - sigma);
        OV_TRY(k_step(c, I, y1, bT.p, m, ek));
        EpiArgs e2;
        e2.m_w = c->m_w;
        e2.s1 = 2.0 * sn / e;
        e2.v[0] = y1;
        e2.w[0] = -2.0 * sn * cc / e;
        e2.v[1] = y0;
        e2.w[1] = -sigma * sn;
        OV_TRY(k_step(c, I, bT.p, y0, m, e2));  // y0 <- new (in place over y_{k-2})
        std::swap(y0, y1);
        sigma = sn;
      }
      Y = y1;
      Z = y0;
    }
    // Rayleigh-Ritz with K^2 in span(Y): G = Y^dag Y, W = K Y, H2 = W^dag W.
    // (Rayleigh-Ritz with the indefinite K itself would produce spurious
    // near-zero Ritz values from mixtures of +lambda and -lambda modes.)
    EpiArgs ek;
    ek.m_w = c->m_w;
    OV_TRY(k_step(c, I, Y, bT.p, m, ek));
    std::vector<cd> G, H2;
    OV_TRY(gram(c, P, Y, m, Y, m, partial, G));
    OV_TRY(gram(c, P, bT.p, m, bT.p, m, partial, H2));
    std::vector<double> th2;
    std::vector<cd> C2;
    rayleigh_ritz(m, G, H2, th2, C2);
    std::vector<double2> C((size_t)m * m);
    for (size_t i = 0; i < C.size(); ++i) C[i] = make_double2(C2[i].real(), C2[i].imag());
    OV_CK(dq.ensure(sizeof(double2) * m * m));
    OV_CK(cudaMemcpyAsync(dq.p, C.data(), sizeof(double2) * m * m, cudaMemcpyHostToDevice, c->st));
    launch_rotate(P, Y, m, dq.as<double2>(), m, Z, V, c->st);  // Z = Y C
    OV_TRY(launched(c));
    launch_rotate(P, bT.p, m, dq.as<double2>(), m, Y, V, c->st);  // Y = (K Y) C
    OV_TRY(launched(c));
    std::swap(Y, Z);  // Y: K^2-Ritz vectors (ascending), Z: K times them
    // Split +lambda / -lambda: Rayleigh-Ritz with K inside the lowest K^2
    // cluster that contains the wanted n_ev vectors.
    int p = n_ev;
    while (p < m && th2[p] - th2[p - 1] < 1e-3 * th2[p - 1]) ++p;
    std::vector<cd> H1;
    OV_TRY(gram(c, P, Y, p, Z, p, partial, H1));
    for (int i = 0; i < p; ++i)
      for (int j = i; j < p; ++j) {
        const cd h = 0.5 * (H1[(size_t)i * p + j] + std::conj(H1[(size_t)j * p + i]));
        H1[(size_t)i * p + j] = h;
        H1[(size_t)j * p + i] = std::conj(h);
      }
    std::vector<double> th;
    std::vector<cd> q;
    herm_eig(p, H1, th, q);
    std::vector<int> ord(p);
    for (int i = 0; i < p; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) {
      const double ax = std::abs(th[x]), ay = std::abs(th[y]);
      return ax != ay ? ax < ay : (th[x] != th[y] ? th[x] < th[y] : x < y);
    });
    std::vector<double2> Q1((size_t)p * p);
    for (int i = 0; i < p; ++i)
      for (int jj = 0; jj < p; ++jj) {
        const cd v = q[(size_t)i * p + ord[jj]];
        Q1[(size_t)i * p + jj] = make_double2(v.real(), v.imag());
      }
    for (int jj = 0; jj < p; ++jj) theta[jj] = th[ord[jj]];
    for (int jj = p; jj < m; ++jj) theta[jj] = std::sqrt(std::max(th2[jj], 0.0));
    OV_CK(cudaMemcpyAsync(dq.p, Q1.data(), sizeof(double2) * p * p, cudaMemcpyHostToDevice, c->st));
    for (void* blk : {Y, Z}) {
      launch_rotate(P, blk, p, dq.as<double2>(), p, bT.p, V, c->st);
      OV_TRY(launched(c));
      OV_CK(cudaMemcpyAsync(blk, bT.p, vb * p, cudaMemcpyDeviceToDevice, c->st));
    }
    // residuals ||K y_j - theta_j y_j||
    double worst = 0.0;
    for (int j = 0; j < n_ev; ++j) {
      launch_axpby(P, 1.0, static_cast<char*>(Z) + j * vb, -theta[j], static_cast<char*>(Y) + j * vb, I.tmp.p, V, 1,
                   c->st);
      OV_TRY(launched(c));
      double r2;
      OV_TRY(norm2(c, P, I.tmp.p, V, &r2));
      res[j] = std::sqrt(r2);
      worst = std::max(worst, res[j]);
    }
    bool finite = std::isfinite(worst);
    for (int j = 0; j < m; ++j) finite = finite && std::isfinite(th2[j]);
    if (!finite) {
      for (DevBuf* b : {&bA, &bB, &bT, &partial, &dq}) b->release();
      return fail(c, OV_ERR_NOT_CONVERGED, "eigensolver: non-finite Ritz values (filter degree too high?)");
    }
    low2 = th2[0];
    cut2 = std::max(th2[m - 1], low2 * 1.0001 + 1e-12);
    if (cut2 >= b2 * 0.999) cut2 = 0.5 * (low2 + b2);
    if (worst <= tol * bmax) {
      converged = true;
      ++iter;
      break;
    }
  }
  c->stats.inner_iterations = iter;  // filter + Rayleigh-Ritz steps taken
  for (int j = 0; j < n_ev; ++j) evals[j] = theta[j];
  if (lambda_max_out) *lambda_max_out = bmax;
  OV_TRY(unpack_output(c, I, Y, evecs, n_ev, OV_C128));
  for (DevBuf* b : {&bA, &bB, &bT, &partial, &dq}) b->release();
  if (!converged) return fail(c, OV_ERR_NOT_CONVERGED, "eigensolver: max_iter reached before tol");
  return OV_OK;
}
