// Stencil instantiations for FP64 storage (see dslash_kernel.cuh).
#include "dslash_kernel.cuh"

namespace ov {

bool launch_dslash_f64(const DslashCfg& c, OpPrec out_prec, const LatticeH& g, const void* links, const void* in,
                      void* out, const EpiArgs& e, int nrhs, cudaStream_t st) {
  (void)out_prec;
  return launch_variant<F64, 18, F64, F64>(c, g, links, in, out, e, nrhs, st);
}

}  // namespace ov
