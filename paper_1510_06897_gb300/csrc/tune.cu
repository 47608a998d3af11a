// Stencil launch shapes: the variant table, the OV_STENCIL pin, the
// autotuner at context creation (one RHS) and per number of right-hand sides
// on first use, and the set-up of an operator instance (link packing, tuning,
// persisting L2 window for 16-bit links).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace ov {

// Times one stencil variant on nrhs right-hand sides: a K step and a
// recurrence step (three extra vector reads), after one warm-up pair; three
// such pairs per run for short launches, one for long ones (several right-
// hand sides, or the ALU-bound FP64 kernel at ~1 ms a launch).
ov_status time_variant(ov_ctx* c, Inst& I, const DslashCfg& cfg, const void* links, int nrhs, DevBuf* buf,
                       cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  EpiArgs ek;
  ek.m_w = c->m_w;
  EpiArgs er = ek;
  er.v[0] = buf[2].p;
  er.w[0] = 0.5;
  er.v[1] = buf[3].p;
  er.w[1] = -1.0;
  er.v[2] = buf[0].p;
  er.w[2] = 0.25;
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) OV_CK(cudaEventRecord(e0, c->st));
    for (int k = 0; k < ((nrhs > 4 || I.p == OP_F64) ? 1 : 3); ++k) {
      if (!launch_dslash(I.p, I.p, cfg, c->g, links, buf[0].p, buf[1].p, ek, nrhs, c->st) ||
          !launch_dslash(I.p, I.p, cfg, c->g, links, buf[1].p, buf[3].p, er, nrhs, c->st))
        return fail(c, OV_ERR_CUDA, "stencil variant not compiled");
    }
    OV_TRY(launched(c, 2));
  }
  OV_CK(cudaEventRecord(e1, c->st));
  OV_CK(cudaEventSynchronize(e1));
  OV_CK(cudaEventElapsedTime(ms, e0, e1));
  return OV_OK;
}

// (minb, rt) pairs compiled for the stencil (see dslash_kernel.cuh).
// (minb 5: <= 64-thread blocks, 14 resident; see dslash_kernel.cuh)
const int kVariants[][2] = {{2, 1}, {3, 1}, {4, 1}, {5, 1}, {2, 2}, {3, 2}, {1, 3}, {2, 3}, {1, 4}, {2, 4}, {1, 6}};

// The environment variable OV_STENCIL="tpb,minb,lrec[,rt[,async[,brick]]]"
// (e.g. "192,3,12" or "64,4,12,1,1") skips the timing and pins one variant
// (used for reproducible profiles; async 1 / 2 selects the shared-memory
// staged kernel for 16-bit storage, register cap minb 3 or 4, 12-real links,
// rt 1; brick 1 maps blocks onto 8 x 4 x (tpb / 32) bricks of sites where the
// lattice allows it);
// OV_STENCIL="slab" pins the slab kernel where it applies (16-bit storage,
// Lx Ly a multiple of 32 up to 640), the default gather variant elsewhere.
bool pinned_cfg(DslashCfg* cfg, bool* bad) {
  *bad = false;
  const char* env = std::getenv("OV_STENCIL");
  if (!env) return false;
  if (std::strcmp(env, "slab") == 0) {
    *cfg = DslashCfg{};
    cfg->slab = 1;  // resolved by the caller
    return true;
  }
  int tpb = 0, minb = 0, lrec = 0, rt = 1, as = 0, bk = 0;
  const int n = std::sscanf(env, "%d,%d,%d,%d,%d,%d", &tpb, &minb, &lrec, &rt, &as, &bk);
  bool ok = n >= 3 && tpb >= 32 && tpb <= 256 && tpb % 32 == 0 && (lrec == 12 || lrec == 18) && as >= 0 && as <= 2 &&
            (bk == 0 || bk == 1) && !(minb >= 5 && tpb > 64);
  bool listed = false;
  for (const auto& v : kVariants) listed = listed || (v[0] == minb && v[1] == rt);
  if (as > 0) listed = (minb == 3 || minb == 4) && rt == 1 && lrec == 12;
  if (!ok || !listed) {
    *bad = true;
    return false;
  }
  *cfg = DslashCfg{tpb, minb, lrec, rt};
  cfg->async = as;
  cfg->brick = bk;
  return true;
}

// The slab kernel's configuration for instance I, if it applies: as many
// persistent CTAs (Lx Ly compute threads + a producer warp) as fit on the SMs.
bool slab_cfg(ov_ctx* c, const Inst& I, DslashCfg* cfg) {
  if (!(I.p == OP_F16 || I.p == OP_B16) || c->d_stencil_err == nullptr || !slab_lattice_ok(c->g)) return false;
  const int per_sm = slab_ctas_per_sm(c->g);
  if (per_sm <= 0) return false;
  *cfg = DslashCfg{};
  cfg->tpb = c->g.L[0] * c->g.L[1] + 32;
  cfg->minb = 1;
  cfg->lrec = 12;
  cfg->slab = c->num_sms * per_sm;
  cfg->err = c->d_stencil_err;
  return true;
}

// Times the one-RHS stencil variants (threads per block, register cap, and
// for 16-bit links the 12- or 18-real layout) on this lattice and keeps the
// fastest; the link layout chosen here is kept for every nrhs.
ov_status autotune(ov_ctx* c, Inst& I, const void* links_dev) {
  const int64_t V = c->g.V;
  I.cfg = DslashCfg{};
  I.cfg_batch.clear();
  const bool is16 = (I.p == OP_F16 || I.p == OP_B16);
  DslashCfg pin;
  bool bad = false;
  const bool pinned = pinned_cfg(&pin, &bad);
  if (bad)
    return fail(c, OV_ERR_INVALID,
                "OV_STENCIL must be \"slab\" or \"tpb,minb,lrec[,rt]\" naming a compiled variant");
  DevBuf alt;  // the other 16-bit link layout
  if (is16 && (!pinned || (pin.slab == 0 && pin.lrec == 18))) {
    OV_CK(alt.ensure((size_t)link_bytes_per_site_dir(I.p, 18) * 4 * V));
    launch_pack_links(I.p, 18, c->g, links_dev, alt.p, c->st);
    OV_TRY(launched(c));
  }
  DslashCfg best_cfg;
  if (pinned && pin.slab) {
    DslashCfg sc;
    if (slab_cfg(c, I, &sc)) best_cfg = sc;
  } else if (pinned) {
    best_cfg = DslashCfg{pin.tpb, pin.minb, is16 ? pin.lrec : 12, 1};
    if (I.p == OP_F64 && pin.rt != 1) best_cfg.rt = 1;
    if (is16) best_cfg.async = pin.async;  // the staged kernel exists for 16-bit storage only
    best_cfg.brick = (pin.brick && brick_lattice_ok(c->g, pin.tpb)) ? 1 : 0;
  } else if (V >= 4096) {
    DevBuf buf[4];
    for (DevBuf& b : buf) {
      OV_CK(b.ensure(I.pbytes(V)));
      OV_CK(cudaMemsetAsync(b.p, 0, I.pbytes(V), c->st));
    }
    cudaEvent_t e0, e1;
    OV_CK(cudaEventCreate(&e0));
    OV_CK(cudaEventCreate(&e1));
    struct Cand {
      float ms;
      DslashCfg cfg;
      const void* links;
    };
    std::vector<Cand> cands;
    for (int lrec : {12, 18}) {
      if (!is16 && lrec == 18) continue;
      const void* links = (lrec == 18 && is16) ? alt.p : I.links.p;
      for (int tpb : {64, 96, 128, 192, 256})
        for (const auto& v : kVariants)
          for (int bk : {0, 1}) {
            if (v[1] != 1 || (bk && !brick_lattice_ok(c->g, tpb)) || (v[0] >= 5 && tpb > 64)) continue;
            DslashCfg cfg{tpb, v[0], is16 ? lrec : 12, 1};
            cfg.brick = bk;
            float ms = 0.f;
            OV_TRY(time_variant(c, I, cfg, links, 1, buf, e0, e1, &ms));
            cands.push_back({ms, cfg, links});
          }
    }
    if (is16) {  // the shared-memory staged kernel (12-real links)
      for (int tpb : {64, 96, 128, 192, 256})
        for (int minb : {3, 4})
          for (int as : {1, 2})
            for (int bk : {0, 1}) {
              if (bk && !brick_lattice_ok(c->g, tpb)) continue;
              DslashCfg cfg{tpb, minb, 12, 1};
              cfg.async = as;
              cfg.brick = bk;
              float ms = 0.f;
              OV_TRY(time_variant(c, I, cfg, I.links.p, 1, buf, e0, e1, &ms));
              cands.push_back({ms, cfg, I.links.p});
            }
    }
    DslashCfg sc;
    if (slab_cfg(c, I, &sc)) {
      float ms = 0.f;
      OV_TRY(time_variant(c, I, sc, I.links.p, 1, buf, e0, e1, &ms));
      cands.push_back({ms, sc, I.links.p});
    }
    // the leaders are often within a few percent: time the best three again,
    // interleaved, and keep each one's fastest run
    std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    const size_t top = std::min<size_t>(3, cands.size());
    for (int rep = 0; rep < 3; ++rep)
      for (size_t k = 0; k < top; ++k) {
        float ms = 0.f;
        OV_TRY(time_variant(c, I, cands[k].cfg, cands[k].links, 1, buf, e0, e1, &ms));
        cands[k].ms = std::min(cands[k].ms, ms);
      }
    size_t win = 0;
    for (size_t k = 1; k < top; ++k)
      if (cands[k].ms < cands[win].ms) win = k;
    if (!cands.empty()) best_cfg = cands[win].cfg;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  I.cfg = best_cfg;
  if (is16 && best_cfg.lrec == 18) std::swap(I.links, alt);
  OV_CK(cudaStreamSynchronize(c->st));
  alt.release();
  return OV_OK;
}

// Stencil shape for nrhs right-hand sides: tuned on first use (threads per
// block, register cap, right-hand sides per thread; link layout as tuned at
// create) and cached per nrhs.  The candidates are timed on at most
// kTuneRhs right-hand sides (one launch of every candidate on all 102 vectors
// of an eigensolver block would cost seconds), which ranks the shapes alike.
constexpr int kTuneRhs = 12;
ov_status batch_cfg(ov_ctx* c, Inst& I, int nrhs, DslashCfg* out) {
  if (nrhs <= 1) {
    *out = I.cfg;
    return OV_OK;
  }
  for (const auto& kv : I.cfg_batch)
    if (kv.first == nrhs) {
      *out = kv.second;
      return OV_OK;
    }
  DslashCfg best_cfg = I.cfg;
  DslashCfg pin;
  bool bad = false;
  if (pinned_cfg(&pin, &bad)) {
    if (!pin.slab) {
      best_cfg = DslashCfg{pin.tpb, pin.minb, I.cfg.lrec, (I.p == OP_F64) ? 1 : pin.rt};
      if (best_cfg.rt == 1 && best_cfg.minb == 1) best_cfg.minb = 2;
      if ((I.p == OP_F16 || I.p == OP_B16) && I.cfg.lrec == 12) best_cfg.async = pin.async;
      best_cfg.brick = (pin.brick && brick_lattice_ok(c->g, pin.tpb)) ? 1 : 0;
    }
  } else if (c->g.V >= 4096) {
    const int64_t V = c->g.V;
    const int nt = std::min(nrhs, kTuneRhs);  // right-hand sides the candidates are timed on
    DevBuf buf[4];
    for (DevBuf& b : buf) {
      OV_CK(b.ensure(I.pbytes(V) * nt));
      OV_CK(cudaMemsetAsync(b.p, 0, I.pbytes(V) * nt, c->st));
    }
    cudaEvent_t e0, e1;
    OV_CK(cudaEventCreate(&e0));
    OV_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int tpb : {64, 96, 128, 192, 256})
      for (const auto& v : kVariants)
        for (int bk : {0, 1}) {
          if (v[1] > nt || (I.p == OP_F64 && v[1] != 1) || (bk && !brick_lattice_ok(c->g, tpb)) ||
              (v[0] >= 5 && tpb > 64))
            continue;
          DslashCfg cfg{tpb, v[0], I.cfg.lrec, v[1]};
          cfg.brick = bk;
          float ms = 0.f;
          OV_TRY(time_variant(c, I, cfg, I.links.p, nt, buf, e0, e1, &ms));
          if (ms < best) {
            best = ms;
            best_cfg = cfg;
          }
        }
    if ((I.p == OP_F16 || I.p == OP_B16) && I.cfg.lrec == 12) {  // the staged kernel, one RHS per thread
      for (int tpb : {64, 96, 128, 192, 256})
        for (int minb : {3, 4})
          for (int as : {1, 2})
            for (int bk : {0, 1}) {
              if (bk && !brick_lattice_ok(c->g, tpb)) continue;
              DslashCfg cfg{tpb, minb, 12, 1};
              cfg.async = as;
              cfg.brick = bk;
              float ms = 0.f;
              OV_TRY(time_variant(c, I, cfg, I.links.p, nt, buf, e0, e1, &ms));
              if (ms < best) {
                best = ms;
                best_cfg = cfg;
              }
            }
    }
    DslashCfg sc;
    if (I.cfg.lrec == 12 && slab_cfg(c, I, &sc)) {
      float ms = 0.f;
      OV_TRY(time_variant(c, I, sc, I.links.p, nt, buf, e0, e1, &ms));
      if (ms < best) {
        best = ms;
        best_cfg = sc;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    OV_CK(cudaStreamSynchronize(c->st));
  }
  I.cfg_batch.emplace_back(nrhs, best_cfg);
  *out = best_cfg;
  return OV_OK;
}

// 16-bit links fit in L2: mark them persisting for the stencil launches
// (a per-process limit, released in ov_destroy).  OV_L2PIN=0 disables.
static ov_status pin_links_in_l2(ov_ctx* c, Inst& I) {
  const char* pin = std::getenv("OV_L2PIN");
  if (!(I.p == OP_F16 || I.p == OP_B16) || (pin && std::atoi(pin) == 0)) return OV_OK;
  const size_t bytes = (size_t)link_bytes_per_site_dir(I.p, I.cfg.lrec) * 4 * c->g.V;
  int dev = 0, max_persist = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) == cudaSuccess &&
      (size_t)max_persist >= bytes && bytes >= (size_t(1) << 20)) {
    OV_CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes));
    l2_window().base = I.links.p;
    l2_window().bytes = bytes;
    c->l2_pinned = true;
  }
  return OV_OK;
}

ov_status init_inst(ov_ctx* c, Inst& I, OpPrec p, const void* links_dev) {
  I.p = p;
  I.pv = (p == OP_F64) ? OP_F64 : OP_F32;
  I.active = true;
  OV_CK(I.links.ensure((size_t)link_bytes_per_site_dir(p, 12) * 4 * c->g.V));
  launch_pack_links(p, 12, c->g, links_dev, I.links.p, c->st);
  OV_TRY(launched(c));
  // the candidates are timed as they will run: 12-real 16-bit links already
  // persisting in L2 (the 18-real copy, timed against them, is not)
  I.cfg.lrec = 12;
  OV_TRY(pin_links_in_l2(c, I));
  OV_TRY(autotune(c, I, links_dev));
  if (c->l2_pinned && l2_window().base != I.links.p) {  // 18-real links won: window over them, if they fit
    l2_window() = L2Window{};
    c->l2_pinned = false;
    OV_TRY(pin_links_in_l2(c, I));
  }
  return OV_OK;
}

}  // namespace ov
