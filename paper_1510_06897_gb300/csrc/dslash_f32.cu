// Stencil instantiations for FP32 storage (see dslash_kernel.cuh).
#include "dslash_kernel.cuh"

namespace ov {

bool launch_dslash_f32(const DslashCfg& c, OpPrec out_prec, const LatticeH& g, const void* links, const void* in,
                      void* out, const EpiArgs& e, int nrhs, cudaStream_t st) {
  (void)out_prec;
  return launch_variant<F32, 12, F32, F32>(c, g, links, in, out, e, nrhs, st);
}

}  // namespace ov
