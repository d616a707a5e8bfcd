// Reduced product in double precision on CUDA cores (the FP64 correctness
// path): Y = A_c B_d with A_c M x Kp and B_d Kp x N, both row-major.
#include "common.hpp"

namespace pj {
namespace {

// A block of 256 threads computes a TILE x TILE block of Y, K' in chunks of TILE
// staged in shared memory; each thread owns TILE * TILE / 256 outputs.  Small
// products take TILE = 16 so that there are enough blocks for the SMs (the
// 256 x 256 output of the FP64 configuration gives 256 blocks instead of 64).
template <int TILE>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                       double* __restrict__ Y, int64_t ldy, int64_t M, int64_t N,
                                                       int64_t K) {
  constexpr int ROWS = 256 / TILE;      // thread rows
  constexpr int PER = TILE / ROWS;      // outputs per thread
  __shared__ double sA[TILE][TILE + 1];
  __shared__ double sB[TILE][TILE + 1];
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  const int64_t i0 = static_cast<int64_t>(blockIdx.y) * TILE, j0 = static_cast<int64_t>(blockIdx.x) * TILE;
  double acc[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) acc[r] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += TILE) {
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int row = ty + ROWS * r;
      sA[row][tx] = (i0 + row < M && k0 + tx < K) ? A[(i0 + row) * K + k0 + tx] : 0.0;
      sB[row][tx] = (k0 + row < K && j0 + tx < N) ? B[(k0 + row) * N + j0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TILE; ++kk) {
      const double b = sB[kk][tx];
#pragma unroll
      for (int r = 0; r < PER; ++r) acc[r] = fma(sA[ty + ROWS * r][kk], b, acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int64_t i = i0 + ty + ROWS * r, j = j0 + tx;
    if (i < M && j < N) Y[i * ldy + j] = acc[r];
  }
}

}  // namespace

cudaError_t launch_gemm_f64(const double* Ac, const double* Bd, double* Y, int64_t ldy, int64_t M, int64_t N,
                            int64_t Kp, cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  int sms = 0;
  if (device_sms(&sms) != PJ_OK) sms = 152;
  if (ceil_div(M, 32) * ceil_div(N, 32) < 2 * sms) {
    dim3 grid(static_cast<unsigned>(ceil_div(N, 16)), static_cast<unsigned>(ceil_div(M, 16)));
    gemm_f64_kernel<16><<<grid, 256, 0, st>>>(Ac, Bd, Y, ldy, M, N, Kp);
  } else {
    dim3 grid(static_cast<unsigned>(ceil_div(N, 32)), static_cast<unsigned>(ceil_div(M, 32)));
    gemm_f64_kernel<32><<<grid, 256, 0, st>>>(Ac, Bd, Y, ldy, M, N, Kp);
  }
  return cudaGetLastError();
}

}  // namespace pj
