// ov_sign_poly_grad: gradient of S = chi^dagger P(K) chi with respect to the
// links, P(K) = K f_N(K^2) the undeflated polynomial of Eq. 3.
//
// Forward: the Clenshaw recurrence b_k = c_k chi + 2 Z b_{k+1} - b_{k+2}
// (k = N..0), g = (b_0 - b_2)/2, S = (K chi)^dagger g, keeping all its terms
// or checkpoints of them (below).  Reverse: with gbar = K chi the adjoint
// vectors obey bbar_0 = gbar/2, bbar_1 = 2 Z bbar_0,
// bbar_2 = 2 Z bbar_1 - bbar_0 - gbar/2, bbar_j = 2 Z bbar_{j-1} - bbar_{j-2},
// and
//   dS = chi^dagger dK g + sum_{k=0}^{N-1} 2 bbar_k^dagger dZ b_{k+1},
//   dZ = alpha (dK K + K dK),
// so each step k contributes the dK pairs (bbar_k, K b_{k+1}) and
// (K bbar_k, b_{k+1}) with weight 2 alpha.  The adjoint runs upward in k
// while the recurrence produced b_k downward.  When the 2N + 1 vectors b_k
// and K b_{k+1} fit in the context's gradient memory allowance (by default
// half the free device memory) the forward sweep writes every one of them to
// its own slot and nothing is recomputed (4N + 3 stencil launches in all);
// otherwise it keeps b_k for k = 1, 2 mod 16 and the reverse sweep recomputes
// b_{k+1} and K b_{k+1} 16 at a time from those checkpoints (6N + ...).
// Either way each segment of 16 adjoint steps folds its 32 pairs into the
// link accumulator with one force launch.
#include "ctx.h"

using namespace ov;

namespace {
constexpr int kSeg = 16;

// Forward Clenshaw sweep b_k = c_k chi + 2 Z b_{k+1} - b_{k+2}, k = N .. 0
// (b_{N+1} = b_{N+2} = 0), Z = alpha K^2 + beta: b_k lands in out_of(k)
// (which must not alias b_{k+1} or b_{k+2}), K b_{k+1} in t_of(k), and
// keep(k, b_k) sees every b_k as it is made.  Returns b_0 and b_2 (b_2 =
// zero when N < 2).
template <class Out, class Tmp, class Keep>
ov_status clenshaw_forward(ov_ctx* c, Inst& I, const std::vector<double>& cf, double alpha, double beta,
                           const void* xchi, const void* zero, Out&& out_of, Tmp&& t_of, void** b0, const void** b2,
                           Keep&& keep) {
  const int N = (int)cf.size() - 1;
  EpiArgs ek;
  ek.m_w = c->m_w;
  const void* bk1 = zero;  // b_{k+1}
  const void* bk2 = zero;  // b_{k+2}
  *b2 = zero;
  for (int k = N; k >= 0; --k) {
    void* out = out_of(k);
    void* t = t_of(k);
    OV_TRY(k_step(c, I, bk1, t, 1, ek));
    EpiArgs e;
    e.m_w = c->m_w;
    e.s1 = 2.0 * alpha;
    e.v[0] = bk1;
    e.w[0] = 2.0 * beta;
    e.v[1] = bk2;
    e.w[1] = -1.0;
    e.v[2] = xchi;
    e.w[2] = cf[k];
    OV_TRY(k_step(c, I, t, out, 1, e));
    OV_TRY(keep(k, out));
    if (k == 2) *b2 = out;
    if (k == 0) *b0 = out;
    bk2 = bk1;
    bk1 = out;
  }
  return OV_OK;
}

// Arguments shared by ov_sign_poly_quad and ov_sign_poly_grad.
ov_status check_poly_args(ov_ctx* c, int order, double lo, double hi, const void* chi, const void* out,
                          ov_dtype dt, const char* name) {
  if (!chi || !out) return fail(c, OV_ERR_INVALID, "null argument");
  if (order < 1) return fail(c, OV_ERR_INVALID, "Chebyshev order must be >= 1");
  if (!(lo > 0.0) || !(hi > lo) || !std::isfinite(hi)) return fail(c, OV_ERR_INVALID, "need 0 < lo < hi");
  OV_TRY(check_dtype(c, 1, dt));
  if (c->prec != OV_FP64 && c->prec != OV_FP32)
    return fail(c, OV_ERR_INVALID, std::string(name) + " needs an OV_FP64 or OV_FP32 context");
  return OV_OK;
}
}  // namespace

// S = chi^dagger P(K) chi = (K chi)^dagger f_N(Z) chi, and optionally P(K) chi.
extern "C" ov_status ov_sign_poly_quad(ov_ctx* c, int order, double lo, double hi, const void* chi, void* p_chi,
                                       ov_dtype dt, double* s_out) {
  if (!c) return OV_ERR_INVALID;
  OV_TRY(check_poly_args(c, order, lo, hi, chi, s_out, dt, "ov_sign_poly_quad"));
  Inst& I = (c->prec == OV_FP64) ? c->hi : c->lo;
  const OpPrec P = I.p;  // == I.pv
  const int64_t V = c->g.V;
  const size_t vb = I.vbytes(V);
  const std::vector<double> cf = chebyshev_coefficients(order, lo, hi);
  const double a2 = lo * lo, b2 = hi * hi;
  const double alpha = 2.0 / (b2 - a2), beta = -(b2 + a2) / (b2 - a2);
  GradWork& w = c->gw;
  DevBuf &xchi = w.xchi, &rot3 = w.rot, &t = w.t, &zero = w.zero, &gvec = w.gvec, &gbar = w.gbar;
  OV_CK(xchi.ensure(vb));
  OV_CK(rot3.ensure(3 * vb));
  OV_CK(t.ensure(vb));
  OV_CK(zero.ensure(vb));
  OV_CK(gvec.ensure(vb));
  OV_CK(gbar.ensure(vb));
  OV_CK(c->d_partial.ensure(sizeof(double2) * kReduceBlocks));
  OV_CK(cudaMemsetAsync(zero.p, 0, vb, c->st));
  OV_TRY(pack_input(c, I, chi, 1, dt, xchi.p));
  void* rot[3] = {rot3.c(), rot3.c() + vb, rot3.c() + 2 * vb};
  void* b0 = nullptr;
  const void* b2v = nullptr;
  OV_TRY(clenshaw_forward(
      c, I, cf, alpha, beta, xchi.p, zero.p, [&](int k) { return rot[k % 3]; }, [&](int) { return t.p; }, &b0, &b2v,
      [](int, void*) { return OV_OK; }));
  launch_axpby(P, 0.5, b0, -0.5, b2v, gvec.p, V, 1, c->st);  // f_N(Z) chi = (b_0 - b_2)/2
  OV_TRY(launched(c));
  EpiArgs ek;
  ek.m_w = c->m_w;
  OV_TRY(k_step(c, I, xchi.p, gbar.p, 1, ek));  // K chi
  double2 s;
  OV_TRY(dots(c, P, gbar.p, gvec.p, V, &s));
  *s_out = s.x;
  if (p_chi != nullptr) {
    OV_TRY(k_step(c, I, gvec.p, t.p, 1, ek));  // P(K) chi = K f_N(Z) chi
    OV_TRY(unpack_output(c, I, t.p, p_chi, 1, dt));
  }
  OV_CK(cudaStreamSynchronize(c->st));
  return OV_OK;
}

extern "C" ov_status ov_sign_poly_grad(ov_ctx* c, int order, double lo, double hi, const void* chi,
                                       void* grad_links, ov_dtype dt) {
  if (!c) return OV_ERR_INVALID;
  OV_TRY(check_poly_args(c, order, lo, hi, chi, grad_links, dt, "ov_sign_poly_grad"));
  Inst& I = (c->prec == OV_FP64) ? c->hi : c->lo;
  const OpPrec P = I.p;  // == I.pv
  const int64_t V = c->g.V;
  const size_t vb = I.vbytes(V);
  const int N = order;
  const std::vector<double> cf = chebyshev_coefficients(N, lo, hi);
  const double a2 = lo * lo, b2 = hi * hi;
  const double alpha = 2.0 / (b2 - a2), beta = -(b2 + a2) / (b2 - a2);

  // every b_k (k = 0..N) and K b_{k+1} (k = 0..N-1) on the device when they
  // fit in the allowance; otherwise checkpoint slots k = 16 j + 1 -> 2 j,
  // k = 16 j + 2 -> 2 j + 1 and segment buffers for the recomputation
  // (vectors this context already holds for it count as free)
  GradWork& w = c->gw;
  size_t allowance;
  if (c->grad_mem < 0) {
    size_t fr = 0, tot = 0;
    OV_CK(cudaMemGetInfo(&fr, &tot));
    allowance = (fr + w.keep.bytes) / 2;
  } else {
    allowance = (size_t)c->grad_mem;
  }
  const bool keep_all = vb * (size_t)(2 * N + 1) <= allowance;
  const int nck = 2 * (N / kSeg + 2);
  DevBuf &xchi = w.xchi, &ck = w.ck, &segb = w.segb, &segt = w.segt, &bbar = w.bbar, &tbar = w.tbar;
  DevBuf &gvec = w.gvec, &gbar = w.gbar, &zero = w.zero, &t = w.t, &G = w.G;
  OV_CK(xchi.ensure(vb));
  if (keep_all) {  // b_k in slots 0..N, K b_{k+1} in slots N+1..2N
    if (w.keep.bytes < vb * (size_t)(2 * N + 1)) {
      OV_CK(cudaStreamSynchronize(c->st));
      w.keep.release();
    }
    OV_CK(w.keep.ensure(vb * (size_t)(2 * N + 1)));
    ck.release();
    segb.release();
    segt.release();
  } else {
    w.keep.release();
    OV_CK(ck.ensure(vb * nck));
    OV_CK(segb.ensure(vb * (kSeg + 2)));
    OV_CK(segt.ensure(vb * (kSeg + 1)));
  }
  OV_CK(bbar.ensure(vb * (kSeg + 2)));
  OV_CK(tbar.ensure(vb * kSeg));
  OV_CK(gvec.ensure(vb));
  OV_CK(gbar.ensure(vb));
  OV_CK(zero.ensure(vb));
  OV_CK(t.ensure(vb));
  const size_t gbytes = (size_t)4 * 9 * V * (P == OP_F64 ? 16 : 8);
  OV_CK(G.ensure(gbytes));
  OV_CK(cudaMemsetAsync(zero.p, 0, vb, c->st));
  OV_CK(cudaMemsetAsync(G.p, 0, gbytes, c->st));
  OV_TRY(pack_input(c, I, chi, 1, dt, xchi.p));
  c->stats.grad_kept_terms = keep_all ? 2 * N + 1 : nck;
  auto slot = [&](DevBuf& b, int i) { return static_cast<void*>(b.c() + (size_t)i * vb); };
  auto Bk = [&](int k) { return slot(w.keep, k); };          // b_k, k = 0..N
  auto Tk = [&](int k) { return slot(w.keep, N + 1 + k); };  // K b_{k+1}, k = 0..N-1
  auto ck_slot = [&](int k) -> void* {
    if (k > N) return zero.p;
    if (k % kSeg == 1) return slot(ck, 2 * (k / kSeg));
    if (k % kSeg == 2) return slot(ck, 2 * (k / kSeg) + 1);
    return nullptr;
  };
  EpiArgs ek;
  ek.m_w = c->m_w;

  // One Clenshaw step: out = c_k chi + 2 alpha K (K bk1) + 2 beta bk1 - bk2 (tk1 = K bk1 kept).
  auto clenshaw = [&](int k, const void* bk1, const void* bk2, void* tk1, void* out) -> ov_status {
    OV_TRY(k_step(c, I, bk1, tk1, 1, ek));
    EpiArgs e;
    e.m_w = c->m_w;
    e.s1 = 2.0 * alpha;
    e.v[0] = bk1;
    e.w[0] = 2.0 * beta;
    e.v[1] = bk2;
    e.w[1] = -1.0;
    e.v[2] = xchi.p;
    e.w[2] = cf[k];
    return k_step(c, I, tk1, out, 1, e);
  };

  // ---- forward sweep: b_k for k = N .. 0, each in its own slot (keep_all) or
  // rotating through three vectors with copies to the checkpoints
  void* b0 = nullptr;
  const void* b2v = nullptr;
  if (keep_all) {
    OV_TRY(clenshaw_forward(
        c, I, cf, alpha, beta, xchi.p, zero.p, [&](int k) { return Bk(k); },
        [&](int k) { return k < N ? Tk(k) : t.p; }, &b0, &b2v, [](int, void*) { return OV_OK; }));
  } else {
    void* rot[3] = {slot(segb, 0), slot(segb, 1), slot(segb, 2)};
    OV_TRY(clenshaw_forward(c, I, cf, alpha, beta, xchi.p, zero.p, [&](int k) { return rot[k % 3]; },
                            [&](int) { return t.p; }, &b0, &b2v, [&](int k, void* bk) -> ov_status {
                              if (void* cs = (k >= 1) ? ck_slot(k) : nullptr)
                                OV_CK(cudaMemcpyAsync(cs, bk, vb, cudaMemcpyDeviceToDevice, c->st));
                              return OV_OK;
                            }));
  }
  // g = (b_0 - b_2)/2 ; gbar = K chi
  launch_axpby(P, 0.5, b0, -0.5, b2v, gvec.p, V, 1, c->st);
  OV_TRY(launched(c));
  OV_TRY(k_step(c, I, xchi.p, gbar.p, 1, ek));

  // ---- reverse sweep, one segment of 16 adjoint steps at a time
  // bbar slots: slot(bbar, k - k0 + 1) holds bbar_k for k in [k0-1, k0+16]
  OV_CK(cudaMemsetAsync(slot(bbar, 0), 0, vb, c->st));  // bbar_{-1} = 0
  launch_axpby(P, 0.5, gbar.p, 0.0, nullptr, slot(bbar, 1), V, 1, c->st);  // bbar_0
  OV_TRY(launched(c));
  bool first_pair = true;
  for (int k0 = 0; k0 < N; k0 += kSeg) {
    const int k1 = std::min(k0 + kSeg, N) - 1;  // last adjoint step of the segment
    if (k0 > 0) {
      OV_CK(cudaMemcpyAsync(slot(bbar, 0), slot(bbar, kSeg), vb, cudaMemcpyDeviceToDevice, c->st));
      OV_CK(cudaMemcpyAsync(slot(bbar, 1), slot(bbar, kSeg + 1), vb, cudaMemcpyDeviceToDevice, c->st));
    }
    // b_{k+1} and K b_{k+1} for the adjoint steps k = k0 .. k1
    auto b_next = [&](int k) { return keep_all ? Bk(k + 1) : slot(segb, k - k0); };
    auto t_next = [&](int k) { return keep_all ? Tk(k) : slot(segt, k - k0); };
    if (!keep_all) {
      // recompute b_j and t_j = K b_j for j = k0+1 .. k1+1 (segb/segt slot j - k0 - 1)
      const int top = k1 + 1;
      // from b_{k0+17}, b_{k0+18} (checkpoints; zero above N) down to b_{k0+1}
      const void* p1 = ck_slot(k0 + kSeg + 1);
      const void* p2 = ck_slot(k0 + kSeg + 2);
      for (int j = k0 + kSeg; j >= k0 + 1; --j) {
        if (j > N) {  // b_j = 0 above the top coefficient
          p2 = p1;
          p1 = zero.p;
          continue;
        }
        void* dst = slot(segb, j - k0 - 1);
        void* tj1 = (j + 1 <= top) ? slot(segt, j - k0) : t.p;
        OV_TRY(clenshaw(j, p1, p2, tj1, dst));
        p2 = p1;
        p1 = dst;
      }
      // t_{k0+1} = K b_{k0+1}
      OV_TRY(k_step(c, I, slot(segb, 0), slot(segt, 0), 1, ek));
    }
    // adjoint steps k = k0 .. k1
    ForcePairs pairs;
    if (first_pair) {
      pairs.u[pairs.n] = xchi.p;
      pairs.v[pairs.n] = gvec.p;
      pairs.w[pairs.n] = 1.0;
      pairs.n++;
      first_pair = false;
    }
    for (int k = k0; k <= k1; ++k) {
      void* bb_k = slot(bbar, k - k0 + 1);
      void* bb_km1 = slot(bbar, k - k0);
      void* tb_k = slot(tbar, k - k0);
      OV_TRY(k_step(c, I, bb_k, tb_k, 1, ek));  // tbar_k = K bbar_k
      pairs.u[pairs.n] = bb_k;
      pairs.v[pairs.n] = t_next(k);  // K b_{k+1}
      pairs.w[pairs.n] = 2.0 * alpha;
      pairs.n++;
      pairs.u[pairs.n] = tb_k;
      pairs.v[pairs.n] = b_next(k);  // b_{k+1}
      pairs.w[pairs.n] = 2.0 * alpha;
      pairs.n++;
      if (k + 1 <= N - 1) {  // bbar_{k+1} = 2 alpha K tbar_k + 2 beta bbar_k - bbar_{k-1} [- gbar/2 at k+1 = 2]
        EpiArgs e;
        e.m_w = c->m_w;
        e.s1 = 2.0 * alpha;
        e.v[0] = bb_k;
        e.w[0] = 2.0 * beta;
        e.v[1] = bb_km1;
        e.w[1] = -1.0;
        if (k + 1 == 2) {
          e.v[2] = gbar.p;
          e.w[2] = -0.5;
        }
        OV_TRY(k_step(c, I, tb_k, slot(bbar, k - k0 + 2), 1, e));
      }
    }
    launch_force_pairs(P, c->g, I.links.p, pairs, G.p, c->st);
    OV_TRY(launched(c));
  }
  void* dout;
  bool staged;
  const size_t obytes = (size_t)4 * V * 9 * 16;
  OV_TRY(stage_out(c, grad_links, obytes, &dout, &staged));
  launch_force_finish(P, G.p, V, dout, c->st);
  OV_TRY(launched(c));
  OV_TRY(finish_out(c, grad_links, obytes, staged));
  return OV_OK;
}

extern "C" ov_status ov_set_grad_memory(ov_ctx* c, long long bytes) {
  if (!c) return OV_ERR_INVALID;
  c->grad_mem = bytes < 0 ? -1 : bytes;
  OV_CK(cudaStreamSynchronize(c->st));
  c->gw.release();
  return OV_OK;
}
