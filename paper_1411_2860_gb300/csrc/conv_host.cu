// proj_conv_host: proj_conv for a signal, templates and output in HOST memory.
//
// The lags are cut into `chunks` consecutive ranges.  Chunk c correlates the
// signal slice s[c Lc .. c Lc + Lc + T - 1) (its projection and correlation are
// those of proj_conv on the slice, so every lag is computed exactly as there)
// into one of two device output buffers, and a second stream copies the
// finished buffer to the host rows of the chunk while the next chunk is being
// computed.  The copy of the result, 4 bytes per (lag, template), is the
// largest cost of a call with host buffers, so hiding the correlation behind
// it shortens the call.
#include "common.hpp"

namespace pj {
namespace {

struct HostLayout {
  int64_t lc;                 // lags per chunk (a multiple of 64)
  int chunks;
  size_t conv_ws, off_sig, off_tpl, off_buf[2], total;
};

pj_status host_layout(int64_t S, int64_t T, int64_t nt, int64_t block, int64_t R, const pj_basis* basis,
                      const pj_precision* prec, int32_t chunks, HostLayout* h) {
  if (chunks < 1 || chunks > 64) return fail(PJ_EINVAL, "chunks=%d must be in [1, 64]", chunks);
  ConvGeom g{};
  PJ_TRY(conv_geom(S, T, nt, block, R, basis, prec, &g));
  const int64_t lags = g.lags;
  int64_t lc = round_up(ceil_div(lags, chunks), 64);
  if (lc > lags) lc = lags;
  h->lc = lc;
  h->chunks = static_cast<int>(ceil_div(lags, lc));
  h->conv_ws = proj_conv_workspace_size(lc + T - 1, T, nt, block, R, basis, prec);
  if (h->conv_ws == 0) return fail(PJ_EINVAL, "invalid chunk geometry");
  size_t off = align_up(h->conv_ws);
  h->off_sig = off;
  off = align_up(off + sizeof(float) * S);
  h->off_tpl = off;
  off = align_up(off + sizeof(float) * nt * T);
  for (int b = 0; b < 2; ++b) {
    h->off_buf[b] = off;
    off = align_up(off + sizeof(float) * lc * nt);
  }
  h->total = off;
  return PJ_OK;
}

// Copies of one chunk may be cut into kCopyWays pieces on as many streams.  On
// the GB300 the copy to host memory ran at about 180 GB/s with one stream or
// two, so one is used.
constexpr int kCopyWays = 1;

// The copy streams and their events, per device and host thread, created on
// first use and kept until the process exits.
struct CopyResources {
  cudaStream_t copy[kCopyWays] = {};
  cudaEvent_t done[2] = {nullptr, nullptr};            // chunk's correlation finished
  cudaEvent_t copied[2][kCopyWays] = {};               // chunk's copies to the host finished
};

pj_status copy_resources(CopyResources** out) {
  static thread_local CopyResources res[64];
  int dev = 0;
  PJ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PJ_ECUDA, "device ordinal %d out of range", dev);
  CopyResources& r = res[dev];
  if (!r.copy[0]) {
    for (int w = 0; w < kCopyWays; ++w) PJ_CUDA_TRY(cudaStreamCreateWithFlags(&r.copy[w], cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      PJ_CUDA_TRY(cudaEventCreateWithFlags(&r.done[b], cudaEventDisableTiming));
      for (int w = 0; w < kCopyWays; ++w)
        PJ_CUDA_TRY(cudaEventCreateWithFlags(&r.copied[b][w], cudaEventDisableTiming));
    }
  }
  *out = &r;
  return PJ_OK;
}

}  // namespace
}  // namespace pj

using namespace pj;

extern "C" {

size_t proj_conv_host_workspace_size(int64_t S, int64_t T, int64_t n_templates, int64_t block, int64_t R,
                                     const pj_basis* basis, const pj_precision* prec, int32_t chunks) {
  HostLayout h{};
  if (host_layout(S, T, n_templates, block, R, basis, prec, chunks, &h) != PJ_OK) return 0;
  return h.total;
}

pj_status proj_conv_host(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                         void* out, int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R,
                         const pj_basis* basis, const pj_precision* prec, int32_t chunks, void* workspace,
                         size_t ws_bytes, void* stream) {
  if (!signal || !templates || !out) return fail(PJ_EINVAL, "signal, templates and out must be non-NULL");
  if (in_dtype != PJ_F32 || out_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "CONV takes and writes PJ_F32");
  HostLayout h{};
  PJ_TRY(host_layout(S, T, n_templates, block, R, basis, prec, chunks, &h));
  if (!workspace) return fail(PJ_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(PJ_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < h.total) return fail(PJ_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, h.total);
  CopyResources* cr = nullptr;
  PJ_TRY(copy_resources(&cr));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* sig = reinterpret_cast<float*>(ws + h.off_sig);
  float* tpl = reinterpret_cast<float*>(ws + h.off_tpl);
  PJ_CUDA_TRY(cudaMemcpyAsync(sig, signal, sizeof(float) * S, cudaMemcpyHostToDevice, st));
  PJ_CUDA_TRY(cudaMemcpyAsync(tpl, templates, sizeof(float) * n_templates * T, cudaMemcpyHostToDevice, st));
  const int64_t lags = S - T + 1;
  for (int c = 0; c < h.chunks; ++c) {
    const int b = c & 1;
    const int64_t m0 = c * h.lc;
    const int64_t n = lags - m0 < h.lc ? lags - m0 : h.lc;
    float* buf = reinterpret_cast<float*>(ws + h.off_buf[b]);
    // the buffer is free once the copies of the chunk before last have left it
    if (c >= 2)
      for (int w = 0; w < kCopyWays; ++w) PJ_CUDA_TRY(cudaStreamWaitEvent(st, cr->copied[b][w], 0));
    PJ_TRY(proj_conv(sig + m0, n + T - 1, tpl, T, n_templates, buf, PJ_F32, PJ_F32, block, R, basis, prec, workspace,
                     h.conv_ws, stream));
    PJ_CUDA_TRY(cudaEventRecord(cr->done[b], st));
    const int64_t piece = ceil_div(n, kCopyWays);
    for (int w = 0; w < kCopyWays; ++w) {
      const int64_t r0 = w * piece, r1 = (w + 1) * piece < n ? (w + 1) * piece : n;
      PJ_CUDA_TRY(cudaStreamWaitEvent(cr->copy[w], cr->done[b], 0));
      if (r1 > r0)
        PJ_CUDA_TRY(cudaMemcpyAsync(static_cast<float*>(out) + (m0 + r0) * n_templates, buf + r0 * n_templates,
                                    sizeof(float) * (r1 - r0) * n_templates, cudaMemcpyDeviceToHost, cr->copy[w]));
      PJ_CUDA_TRY(cudaEventRecord(cr->copied[b][w], cr->copy[w]));
    }
  }
  // The caller's stream completes only after every copy to the host has.
  for (int b = 0; b < 2 && b < h.chunks; ++b)
    for (int w = 0; w < kCopyWays; ++w) PJ_CUDA_TRY(cudaStreamWaitEvent(st, cr->copied[b][w], 0));
  return PJ_OK;
}

}  // extern "C"
