// Context helpers shared by the host files of the library: error and launch
// accounting, host/device staging of caller vectors, stencil launches with
// optional profiling, FP64 reductions read back to the host, work buffers and
// the interface pack / unpack.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace ov {

ov_status fail(ov_ctx* c, ov_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ov_status launched(ov_ctx* c, int n) {
  c->stats.kernel_launches += n;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, OV_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return OV_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller input: the pointer itself, or a staged copy.
ov_status stage_in(ov_ctx* c, DevBuf& buf, const void* p, size_t bytes, const void** out) {
  if (is_device_ptr(p)) {
    *out = p;
    return OV_OK;
  }
  OV_CK(buf.ensure(bytes));
  OV_CK(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, c->st));
  *out = buf.p;
  return OV_OK;
}

// Device destination for a caller output; finish_out copies it back if needed.
ov_status stage_out(ov_ctx* c, void* p, size_t bytes, void** out, bool* staged) {
  if (is_device_ptr(p)) {
    *out = p;
    *staged = false;
    return OV_OK;
  }
  OV_CK(c->stage_out.ensure(bytes));
  *out = c->stage_out.p;
  *staged = true;
  return OV_OK;
}

// After a stream sync: a slab stencil launch whose bulk copies did not land
// in time left its flag set.
ov_status stencil_status(ov_ctx* c) {
  if (c->h_stencil_err && *static_cast<volatile int*>(c->h_stencil_err)) {
    *c->h_stencil_err = 0;
    return fail(c, OV_ERR_CUDA, "stencil: a shared-memory bulk copy did not complete in time");
  }
  return OV_OK;
}

ov_status finish_out(ov_ctx* c, void* host, size_t bytes, bool staged) {
  if (staged) OV_CK(cudaMemcpyAsync(host, c->stage_out.p, bytes, cudaMemcpyDeviceToHost, c->st));
  OV_CK(cudaStreamSynchronize(c->st));
  prof_collect(c);
  return stencil_status(c);
}

void prof_collect(ov_ctx* c) {
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->evs[i], c->evs[i + 1]) == cudaSuccess) {
      c->stats.dslash_ms += ms;
      c->stats.dslash_timed += c->ev_count[i / 2];
    } else {
      cudaGetLastError();
    }
  }
  c->ev_used = 0;
}

ov_status prof_open(ov_ctx* c) {
  while (c->evs.size() < c->ev_used + 2) {
    cudaEvent_t ev;
    OV_CK(cudaEventCreate(&ev));
    c->evs.push_back(ev);
  }
  if (c->ev_count.size() < c->evs.size() / 2) c->ev_count.resize(c->evs.size() / 2);
  OV_CK(cudaEventRecord(c->evs[c->ev_used], c->st));
  return OV_OK;
}

ov_status prof_close(ov_ctx* c, int n) {
  OV_CK(cudaEventRecord(c->evs[c->ev_used + 1], c->st));
  c->ev_count[c->ev_used / 2] = n;
  c->ev_used += 2;
  return OV_OK;
}

ov_status dslash(ov_ctx* c, Inst& I, OpPrec out_prec, const void* in, void* out, const EpiArgs& e, int nrhs) {
  DslashCfg cfg;
  OV_TRY(batch_cfg(c, I, nrhs, &cfg));
  if (c->stall_cycles > 0) {
    cfg.stall = c->d_never.as<int>();
    cfg.stall_cycles = c->stall_cycles;
  }
  if (c->prof == 1) OV_TRY(prof_open(c));
  if (!launch_dslash(I.p, out_prec, cfg, c->g, I.links.p, in, out, e, nrhs, c->st))
    return fail(c, OV_ERR_CUDA, "stencil variant not compiled");
  c->stats.dslash_launches++;
  ov_status s = launched(c);
  if (s != OV_OK) return s;
  if (c->prof == 1) OV_TRY(prof_close(c, 1));
  return OV_OK;
}

size_t iface_bytes(const LatticeH& g, int nrhs, ov_dtype dt) {
  return (size_t)g.V * nrhs * 12 * (dt == OV_C128 ? 16 : 8);
}

ov_status ensure_scalars(ov_ctx* c, int n) {
  if (c->h_scalars_n < n) {
    if (c->h_scalars) cudaFreeHost(c->h_scalars);
    c->h_scalars = nullptr;
    c->h_scalars_n = 0;
    OV_CK(cudaMallocHost(&c->h_scalars, sizeof(double2) * n));
    c->h_scalars_n = n;
  }
  OV_CK(c->d_scalars.ensure(sizeof(double2) * n));
  return OV_OK;
}

// Reads back n double2 values reduced from partial sums.
ov_status read_reduced(ov_ctx* c, const double2* partial, int n, double2* out) {
  OV_TRY(ensure_scalars(c, n));
  launch_reduce_partials(partial, n, kReduceBlocks, c->d_scalars.as<double2>(), c->st);
  OV_TRY(launched(c));
  OV_CK(cudaMemcpyAsync(c->h_scalars, c->d_scalars.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->st));
  OV_CK(cudaStreamSynchronize(c->st));
  prof_collect(c);
  OV_TRY(stencil_status(c));
  std::memcpy(out, c->h_scalars, sizeof(double2) * n);
  return OV_OK;
}

ov_status ensure_work(ov_ctx* c, Inst& I, int nrhs) {
  const int64_t V = c->g.V;
  const size_t vb = I.vbytes(V) * nrhs, pb = I.pbytes(V) * nrhs;
  OV_CK(I.xin.ensure(vb));
  OV_CK(I.xout.ensure(vb));
  OV_CK(I.d.ensure(vb));
  OV_CK(I.tmp.ensure(vb));
  OV_CK(I.perp.ensure(pb));
  OV_CK(I.t.ensure(pb));
  OV_CK(I.bA.ensure(pb));
  OV_CK(I.bB.ensure(pb));
  OV_CK(c->d_partial.ensure(sizeof(double2) * kReduceBlocks * (size_t)std::max(1, c->n_ev)));
  OV_CK(c->d_c.ensure(sizeof(double2) * (size_t)std::max(1, c->n_ev) * nrhs));
  return OV_OK;
}

ov_status dots(ov_ctx* c, OpPrec p, const void* a, const void* b, int64_t V, double2* out) {
  launch_dot_partial(p, a, b, V, 1, c->d_partial.as<double2>(), c->st);
  OV_TRY(launched(c));
  return read_reduced(c, c->d_partial.as<double2>(), 1, out);
}

ov_status norm2(ov_ctx* c, OpPrec p, const void* a, int64_t V, double* out) {
  launch_norm2_partial(p, a, V, 1, c->d_partial.as<double2>(), c->st);
  OV_TRY(launched(c));
  double2 r;
  OV_TRY(read_reduced(c, c->d_partial.as<double2>(), 1, &r));
  *out = r.x;
  return OV_OK;
}

ov_status check_dtype(ov_ctx* c, int nrhs, ov_dtype dt) {
  if (nrhs < 1) return fail(c, OV_ERR_INVALID, "nrhs must be >= 1");
  if (nrhs > 65535) return fail(c, OV_ERR_INVALID, "nrhs must be <= 65535 (one stencil grid slot each)");
  if (dt != OV_C128 && dt != OV_C64) return fail(c, OV_ERR_INVALID, "dtype must be OV_C128 or OV_C64");
  return OV_OK;
}

ov_status pack_input(ov_ctx* c, Inst& I, const void* in, int nrhs, ov_dtype dt, void* dst) {
  const void* din;
  OV_TRY(stage_in(c, c->stage_in, in, iface_bytes(c->g, nrhs, dt), &din));
  launch_pack_spinor(I.pv, dt == OV_C128 ? IF_C128 : IF_C64, c->g, din, dst, nrhs, 1.0, 0, c->st);
  return launched(c);
}

ov_status unpack_output(ov_ctx* c, Inst& I, const void* src, void* out, int nrhs, ov_dtype dt) {
  if (c->checks) {  // a NaN or Inf anywhere makes the sum of squares non-finite
    launch_norm2_partial(I.pv, src, c->g.V, nrhs, c->d_partial.as<double2>(), c->st);
    OV_TRY(launched(c));
    double2 n2;
    OV_TRY(read_reduced(c, c->d_partial.as<double2>(), 1, &n2));
    if (!std::isfinite(n2.x)) return fail(c, OV_ERR_NONFINITE, "output holds NaN or Inf values (checks are on)");
  }
  void* dout;
  bool staged;
  const size_t bytes = iface_bytes(c->g, nrhs, dt);
  OV_TRY(stage_out(c, out, bytes, &dout, &staged));
  launch_unpack_spinor(I.pv, dt == OV_C128 ? IF_C128 : IF_C64, c->g, src, dout, nrhs, 1.0, c->st);
  OV_TRY(launched(c));
  return finish_out(c, out, bytes, staged);
}

}  // namespace ov
