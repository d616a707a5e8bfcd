// Failure-detection self-test: kernels whose bounded waits cannot be satisfied,
// so that a test can check, on the GPU, that a wait gives up after its limit,
// records its code in the workspace's error word, that the kernel drains what
// it issued and exits, and that the context stays usable (no trap, no fault,
// no hang).  The paper has no counterpart.
#include "common.hpp"
#include "tc.cuh"

namespace pj {
namespace {

// Thread 0 waits on an mbarrier that nothing arrives at and gives up after the
// wait limit; thread 32 waits on the same phase and gives up as soon as the
// error word is set (the path every other waiting warp of a failed kernel takes).
__global__ void wait_selftest_kernel(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 || threadIdx.x == 32) mbar_wait(&bar, 0, err, DEV_TIMEOUT_SELFTEST);
}

// The product of the GEMM self-test: 256 x 256 output, reduced dimension 1024
// (16 K stages of BF16), two tile columns, so it runs on one CTA pair (on two
// solo CTAs in the build without pairs).
constexpr int64_t kSelfM = 256, kSelfN = 256, kSelfK = 1024;
constexpr size_t kSelfQ = kHeaderBytes;
constexpr size_t kSelfP = kSelfQ + kSelfM * kSelfK * 2;
constexpr size_t kSelfY = kSelfP + kSelfN * kSelfK * 2;
constexpr size_t kSelfBytes = kSelfY + kSelfM * kSelfN * 4;

}  // namespace
}  // namespace pj

using namespace pj;

extern "C" {

size_t pj_selftest_workspace_size(void) { return align_up(kSelfBytes); }

pj_status pj_selftest_timeout(int32_t which, void* workspace, size_t ws_bytes, void* stream) {
  if (which != 0 && which != 1) return fail(PJ_EINVAL, "which=%d must be 0 or 1", which);
  PJ_TRY(check_ws(workspace, ws_bytes, pj_selftest_workspace_size()));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  if (which == 0) {
    wait_selftest_kernel<<<1, 64, 0, st>>>(error_word(workspace));
    PJ_CUDA_TRY(cudaGetLastError());
    return PJ_OK;
  }
  char* ws = static_cast<char*>(workspace);
  PJ_CUDA_TRY(cudaMemsetAsync(ws + kSelfQ, 0, kSelfY - kSelfQ, st));
  GemmTcArgs a;
  a.Q = reinterpret_cast<const uint16_t*>(ws + kSelfQ);
  a.ldq = kSelfK;
  a.rowsQ = kSelfM;
  a.P = reinterpret_cast<const uint16_t*>(ws + kSelfP);
  a.ldp = kSelfK;
  a.rowsP = kSelfN;
  a.xdim = kSelfK;
  a.kdim = kSelfK;
  a.nseg = 1;
  a.segQ[0] = a.segP[0] = 0;
  a.Y = ws + kSelfY;
  a.ldy = kSelfN;
  a.out_dtype = PJ_F32;
  a.stall_stage = 2;  // both producers of the pair stop after two of the 16 stages
  PJ_CUDA_TRY(launch_gemm_tc_generic(a, error_word(workspace), sms, st));
  return PJ_OK;
}

}  // extern "C"
