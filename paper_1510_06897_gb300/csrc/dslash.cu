// Stencil dispatch: picks the per-precision launcher compiled in
// dslash_f64.cu / dslash_f32.cu / dslash_f16.cu / dslash_b16.cu.
#include "dslash_kernel.cuh"

namespace ov {

L2Window& l2_window() {
  static L2Window w;
  return w;
}

bool launch_dslash_f64(const DslashCfg&, OpPrec, const LatticeH&, const void*, const void*, void*, const EpiArgs&, int,
                       cudaStream_t);
bool launch_dslash_f32(const DslashCfg&, OpPrec, const LatticeH&, const void*, const void*, void*, const EpiArgs&, int,
                       cudaStream_t);
bool launch_dslash_f16(const DslashCfg&, OpPrec, const LatticeH&, const void*, const void*, void*, const EpiArgs&, int,
                       cudaStream_t);
bool launch_dslash_b16(const DslashCfg&, OpPrec, const LatticeH&, const void*, const void*, void*, const EpiArgs&, int,
                       cudaStream_t);

bool launch_dslash(OpPrec p, OpPrec out_prec, const DslashCfg& cfg, const LatticeH& g, const void* links,
                   const void* in, void* out, const EpiArgs& e, int nrhs, cudaStream_t st) {
  switch (p) {
    case OP_F64: return launch_dslash_f64(cfg, out_prec, g, links, in, out, e, nrhs, st);
    case OP_F32: return launch_dslash_f32(cfg, out_prec, g, links, in, out, e, nrhs, st);
    case OP_F16: return launch_dslash_f16(cfg, out_prec, g, links, in, out, e, nrhs, st);
    case OP_B16: return launch_dslash_b16(cfg, out_prec, g, links, in, out, e, nrhs, st);
  }
  return false;
}

}  // namespace ov
