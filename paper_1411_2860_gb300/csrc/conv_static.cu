// proj_conv_noalloc: the projected cross-correlation of proj_conv for callers
// that cannot allocate device memory.  A plug-in living inside a host
// application that owns the device allocator, or a latency-critical loop that
// must not call cudaMalloc (which may synchronize the whole device), has no
// way to provide the workspace proj_conv asks for.  This entry point uses a
// fixed scratch area instead: a file-scope device array of kStaticScratchBytes
// that exists on every GPU that loads this part of the library, until the
// process exits.  It performs no allocation of its own.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.hpp"

namespace pj {
namespace {

// 20 MiB: enough for a 2^20-sample signal with up to 64 templates of 4096 at
// full R (about 18 MB of projected signal, template chunks and header).
constexpr size_t kStaticScratchBytes = size_t(20) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The array's device address belongs to one CUDA context (the module instance
// loaded into it).  It is cached per context, keyed by the context's unique ID
// (cuCtxGetId): after cudaDeviceReset, or with another context current on the
// same device, the ID differs and the address is looked up again, so a cached
// address of a destroyed context is never used.
struct AddrEntry {
  unsigned long long ctx_id;
  void* addr;
};
constexpr int kAddrCache = 64;
std::mutex g_addr_mu;
AddrEntry g_addr[kAddrCache];
int g_addr_n = 0, g_addr_next = 0;

// Driver calls reached through the runtime's entry-point query, so the library
// does not link libcuda directly.
struct CtxFns {
  PFN_cuCtxGetCurrent_v4000 current = nullptr;
  PFN_cuCtxGetId_v12000 id = nullptr;
};
const CtxFns& ctx_fns() {
  static const CtxFns f = [] {
    CtxFns r;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      r.current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      r.id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    return r;
  }();
  return f;
}

// Device address of the scratch array in the current context: looked up
// (cudaGetSymbolAddress, with that context current) on the first call in each
// context, then taken from the cache.  In host code the array's name is only a
// stand-in, never a device address.
pj_status static_scratch(void** out) {
  int dev = 0;
  PJ_CUDA_TRY(cudaGetDevice(&dev));
  // make the device's primary context current (created here if this thread has none yet)
  PJ_CUDA_TRY(cudaSetDevice(dev));
  const CtxFns& f = ctx_fns();
  if (!f.current || !f.id) return fail(PJ_ECUDA, "cuCtxGetCurrent / cuCtxGetId are not available");
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (f.current(&ctx) != CUDA_SUCCESS || !ctx || f.id(ctx, &id) != CUDA_SUCCESS)
    return fail(PJ_ECUDA, "no current CUDA context on device %d", dev);
  std::lock_guard<std::mutex> lock(g_addr_mu);
  for (int i = 0; i < g_addr_n; ++i)
    if (g_addr[i].ctx_id == id) {
      *out = g_addr[i].addr;
      return PJ_OK;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
  AddrEntry& slot = g_addr_n < kAddrCache ? g_addr[g_addr_n++] : g_addr[g_addr_next++ % kAddrCache];
  slot.ctx_id = id;
  slot.addr = p;
  *out = p;
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
