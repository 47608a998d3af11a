// Stencil instantiations for F16 storage (see dslash_kernel.cuh).
#include "dslash_async.cuh"
#include "dslash_slab.cuh"

namespace ov {

bool launch_dslash_f16(const DslashCfg& c, OpPrec out_prec, const LatticeH& g, const void* links, const void* in,
                      void* out, const EpiArgs& e, int nrhs, cudaStream_t st) {
  if (c.slab > 0) {
    if (c.lrec != 12) return false;
    const bool done = (out_prec == OP_F32) ? launch_slab<F16, F32>(c, g, links, in, out, e, nrhs, st)
                                           : launch_slab<F16, F16>(c, g, links, in, out, e, nrhs, st);
    if (done) return true;
    // an epilogue or pointer the slab kernel does not take: the default gather variant
    const DslashCfg d{};
    if (out_prec == OP_F32) return launch_variant<F16, 12, F16, F32>(d, g, links, in, out, e, nrhs, st);
    return launch_variant<F16, 12, F16, F16>(d, g, links, in, out, e, nrhs, st);
  }
  if (c.async > 0) {
    return (out_prec == OP_F32) ? launch_async<F16, F32>(c, g, links, in, out, e, nrhs, st)
                                : launch_async<F16, F16>(c, g, links, in, out, e, nrhs, st);
  }
  if (out_prec == OP_F32) {
    if (c.lrec == 18) return launch_variant<F16, 18, F16, F32>(c, g, links, in, out, e, nrhs, st);
    return launch_variant<F16, 12, F16, F32>(c, g, links, in, out, e, nrhs, st);
  }
  if (c.lrec == 18) return launch_variant<F16, 18, F16, F16>(c, g, links, in, out, e, nrhs, st);
  return launch_variant<F16, 12, F16, F16>(c, g, links, in, out, e, nrhs, st);
}

}  // namespace ov
