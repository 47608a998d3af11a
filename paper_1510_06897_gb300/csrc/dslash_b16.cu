// Stencil instantiations for B16 storage (see dslash_kernel.cuh).
#include "dslash_kernel.cuh"

namespace ov {

bool launch_dslash_b16(const DslashCfg& c, OpPrec out_prec, const LatticeH& g, const void* links, const void* in,
                      void* out, const EpiArgs& e, int nrhs, cudaStream_t st) {
  if (out_prec == OP_F32) {
    if (c.lrec == 18) return launch_variant<B16, 18, B16, F32>(c, g, links, in, out, e, nrhs, st);
    return launch_variant<B16, 12, B16, F32>(c, g, links, in, out, e, nrhs, st);
  }
  if (c.lrec == 18) return launch_variant<B16, 18, B16, B16>(c, g, links, in, out, e, nrhs, st);
  return launch_variant<B16, 12, B16, B16>(c, g, links, in, out, e, nrhs, st);
}

}  // namespace ov
