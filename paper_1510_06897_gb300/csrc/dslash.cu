// Stencil dispatch: picks the per-precision launcher compiled in
// dslash_f64.cu / dslash_f32.cu / dslash_f16.cu / dslash_b16.cu.
#include <cstdlib>

#include "dslash_slab.cuh"

namespace ov {

bool slab_lattice_ok(const LatticeH& g) { return slab_supported(g); }

int slab_ctas_per_sm(const LatticeH& g) {
  if (!slab_supported(g)) return 0;
  const int P = g.L[0] * g.L[1];
  const size_t smem = slab::slab_smem_bytes(P);
  auto kern = slab::k_dslash_slab<F16, F16>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, P + 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* env = std::getenv("OV_PDL");
    return !(env && std::atoi(env) == 0);
  }();
  return on;
}

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
