// ov_wilson_noalloc: D_W (FP64) for callers that must not allocate device
// memory, e.g. code running inside a framework whose memory pool owns the
// whole device, or a time-critical loop where a cudaMalloc could block or
// fail.  It is the ov_wilson path of an OV_FP64 context (links and spinors
// packed into the stencil's SoA layout, one stencil launch, unpack), except
// that the packed copies live in one fixed file-scope device array instead
// of memory allocated per context.  The caller passes the links, the input
// and the output in device memory; nothing else is needed.
//
// Limits and sharing:
//   * the array holds kNoallocScratchBytes (32 MiB); a call needs
//     V * (4*144 + 2*192*nrhs) bytes and is rejected with OV_ERR_INVALID
//     beyond that (e.g. V <= 34952 sites for one right-hand side);
//   * every GPU that loads this library keeps the array until the process
//     exits;
//   * all calls share the one array and it keeps the contents of the last
//     call: calls that can overlap on the GPU (different streams, or host
//     threads racing) race on it and must be serialised by the caller.  Every
//     byte a call reads from the array is written earlier in the same call,
//     so nothing has to be cleared between calls.
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/overlap.h"
#include "internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

}  // namespace

namespace ov {
void set_thread_error(const std::string& msg);  // read back by ov_last_error(NULL)
}

namespace {

ov_status noalloc_fail(ov_status s, const std::string& msg) {
  ov::set_thread_error(msg);
  return s;
}

// Device address of the scratch array on the current device (looked up once).
ov_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(OV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(OV_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return noalloc_fail(OV_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return OV_OK;
}

// Device (or managed) memory that the current device can use: a device
// pointer of another GPU is refused, since the kernels would run on the
// current device against memory it may not be able to reach.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

extern "C" ov_status ov_wilson_noalloc(const int dims[4], const void* links, const void* in, void* out, int nrhs,
                                       ov_dtype dtype, int antiperiodic_t, void* cuda_stream) {
  using namespace ov;
  set_thread_error("");
  if (!dims || !links || !in || !out) return noalloc_fail(OV_ERR_INVALID, "null argument");
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2) return noalloc_fail(OV_ERR_INVALID, "every lattice extent must be >= 2");
    V *= dims[i];
  }
  if (nrhs < 1) return noalloc_fail(OV_ERR_INVALID, "nrhs must be >= 1");
  if (dtype != OV_C128 && dtype != OV_C64) return noalloc_fail(OV_ERR_INVALID, "dtype must be OV_C128 or OV_C64");
  const size_t link_bytes = align256((size_t)link_bytes_per_site_dir(OP_F64) * 4 * (size_t)V);
  const size_t vec_bytes = align256((size_t)spinor_bytes_per_site(OP_F64) * (size_t)V * (size_t)nrhs);
  if (V > (1LL << 27) || link_bytes + 2 * vec_bytes > kNoallocScratchBytes)
    return noalloc_fail(OV_ERR_INVALID, "lattice x nrhs too large for the 32 MiB scratch of ov_wilson_noalloc: needs " +
                                            std::to_string(link_bytes + 2 * vec_bytes) + " bytes");
  int cur = 0;
  const cudaError_t de = cudaGetDevice(&cur);
  if (de != cudaSuccess) return noalloc_fail(OV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(de));
  if (!on_device(links, cur) || !on_device(in, cur) || !on_device(out, cur))
    return noalloc_fail(OV_ERR_INVALID, "links, in and out must be device memory of the current device");
  void* base = nullptr;
  ov_status s = scratch_address(&base);
  if (s != OV_OK) return s;
  char* scratch = static_cast<char*>(base);
  void* packed_links = scratch;
  void* packed_in = scratch + link_bytes;
  void* packed_out = scratch + link_bytes + vec_bytes;

  LatticeH g;
  for (int i = 0; i < 4; ++i) g.L[i] = dims[i];
  g.V = V;
  g.antiperiodic_t = antiperiodic_t ? 1 : 0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const IfaceType it = (dtype == OV_C128) ? IF_C128 : IF_C64;
  launch_pack_links(OP_F64, 18, g, links, packed_links, st);
  launch_pack_spinor(OP_F64, it, g, in, packed_in, nrhs, 1.0, 0, st);
  EpiArgs e;
  e.wilson = 1;
  DslashCfg cfg;
  launch_dslash(OP_F64, OP_F64, cfg, g, packed_links, packed_in, packed_out, e, nrhs, st);
  launch_unpack_spinor(OP_F64, it, g, packed_out, out, nrhs, 1.0, st);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return noalloc_fail(OV_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(ce));
  ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return noalloc_fail(OV_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(ce));
  return OV_OK;
}
