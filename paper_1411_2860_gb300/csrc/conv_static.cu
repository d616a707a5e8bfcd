// proj_conv_noalloc: the projected cross-correlation of proj_conv for callers
// that cannot allocate device memory.  A plug-in living inside a host
// application that owns the device allocator, or a latency-critical loop that
// must not call cudaMalloc (which may synchronize the whole device), has no
// way to provide the workspace proj_conv asks for.  This entry point uses a
// fixed scratch area instead: a file-scope device array of kStaticScratchBytes
// that exists on every GPU that loads this part of the library, until the
// process exits.  It performs no allocation of its own.
#include <mutex>

#include "common.hpp"

namespace pj {
namespace {

// 20 MiB: enough for a 2^20-sample signal with up to 64 templates of 4096 at
// full R (about 18 MB of projected signal, template chunks and header).
constexpr size_t kStaticScratchBytes = size_t(20) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
void* g_addr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).  In host code
// the array's name is only a stand-in, never a device address.
pj_status static_scratch(void** out) {
  int dev = 0;
  PJ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PJ_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return PJ_OK;
}

}  // namespace
}  // namespace pj

using namespace pj;

extern "C" pj_status proj_conv_noalloc(const void* signal, int64_t S, const void* templates, int64_t T,
                                       int64_t n_templates, void* out, int32_t in_dtype, int32_t out_dtype,
                                       int64_t block, int64_t R, const pj_basis* basis, const pj_precision* prec,
                                       void* stream) {
  const size_t need = proj_conv_workspace_size(S, T, n_templates, block, R, basis, prec);
  if (need == 0)  // invalid or unsupported arguments: let proj_conv name the problem
    return proj_conv(signal, S, templates, T, n_templates, out, in_dtype, out_dtype, block, R, basis, prec,
                     nullptr, 0, stream);
  if (need > kStaticScratchBytes)
    return fail(PJ_ENOMEM, "proj_conv_noalloc: this problem needs %zu bytes of scratch, the static area holds %zu "
                           "(20 MiB); use proj_conv with a workspace",
                need, kStaticScratchBytes);
  void* ws = nullptr;
  PJ_TRY(static_scratch(&ws));
  // proj_conv clears the error word itself and overwrites every other byte it reads.
  return proj_conv(signal, S, templates, T, n_templates, out, in_dtype, out_dtype, block, R, basis, prec, ws,
                   kStaticScratchBytes, stream);
}
