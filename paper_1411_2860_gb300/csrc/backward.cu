// Kernels of the projected-GEMM gradients.  With Y = A P B and
// P = blockdiag(C_R D_R) (Sec. III-B; Eq. 15 truncated as in Eq. 8):
//   dA = dY (P B)^T = expand_C(dY B_d^T),   dB = (A P)^T dY = expand_D(A_c^T dY)
// where B_d, A_c are the projected operands (recomputed, not stored) and the
// expansions map components back to samples:
//   expand_C(X)[i][gL+t] = sum_p X[i][(g,p)] c[t,p],
//   expand_D(X)[gL+t][j] = sum_p d[p,t] X[(g,p)][j].
// The two reduced products run on the tcgen05 GEMM (BF16) or the FP64 kernel.
#include <cuda_bf16.h>

#include "common.hpp"

namespace pj {
namespace {

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ void store(float* p, float v) { *p = v; }
__device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store(double* p, double v) { *p = v; }

// Component p of global group gg (L consecutive inner-dimension values) is
// column gg * (l+1) + p of the reduced inner dimension.
struct Groups {
  int64_t K;
  int L, lp1;
  __device__ __forceinline__ int count(int64_t gg) const {
    const int64_t rem = K - gg * L;
    return static_cast<int>(rem < L ? rem : L);
  }
};

// B (K x N) -> B_d (Kp x N, pitch ldo) in BF16, not transposed; one thread per
// (group, column), coalesced along the columns.
template <typename InT>
__global__ void __launch_bounds__(256) project_cols_nt_kernel(const InT* __restrict__ B, int64_t ldb, int64_t N,
                                                              Groups gr, const float* __restrict__ Ds,
                                                              uint16_t* __restrict__ Bd, int64_t ldo) {
  const int64_t gg = blockIdx.x;
  const int64_t j = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int n = gr.count(gg);
  float x[64];
  for (int t = 0; t < gr.L; ++t) x[t] = t < n ? to_float(B[(gg * gr.L + t) * ldb + j]) : 0.0f;
  for (int p = 0; p < gr.lp1; ++p) {
    float acc = 0.0f;
    for (int t = 0; t < gr.L; ++t) acc = fmaf(Ds[p * gr.L + t], x[t], acc);
    Bd[(gg * gr.lp1 + p) * ldo + j] = __bfloat16_as_ushort(__float2bfloat16_rn(acc));
  }
}

// X (rows x cols, pitch ldx) -> BF16 transpose (cols x rows, pitch ldo) via 32 x 32 tiles.
template <typename InT>
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const InT* __restrict__ X, int64_t ldx, int64_t rows,
                                                             int64_t cols, uint16_t* __restrict__ out,
                                                             int64_t ldo) {
  __shared__ float tile[32][33];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = r0 + k, c = c0 + tx;
    tile[k][tx] = (r < rows && c < cols) ? to_float(X[r * ldx + c]) : 0.0f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t c = c0 + k, r = r0 + tx;
    if (c < cols && r < rows) out[c * ldo + r] = __bfloat16_as_ushort(__float2bfloat16_rn(tile[tx][k]));
  }
}

// X (rows x cols, pitch ldx) -> BF16 copy (pitch ldo).
template <typename InT>
__global__ void __launch_bounds__(256) convert_bf16_kernel(const InT* __restrict__ X, int64_t ldx, int64_t rows,
                                                           int64_t cols, uint16_t* __restrict__ out, int64_t ldo) {
  const int64_t c = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  const int64_t r = blockIdx.x;
  if (c < cols && r < rows) out[r * ldo + c] = __bfloat16_as_ushort(__float2bfloat16_rn(to_float(X[r * ldx + c])));
}

// dA[i][gg*L + t] = sum_p X[i][(g,p)] c[t,p]  (X: M x Kp, pitch ldx)
template <typename AccT, typename OutT>
__global__ void __launch_bounds__(256) expand_rows_kernel(const AccT* __restrict__ X, int64_t ldx, int64_t M,
                                                          Groups gr, int64_t NG, const AccT* __restrict__ Cs,
                                                          OutT* __restrict__ dA, int64_t ldda) {
  const int64_t i = blockIdx.x;
  const int64_t gg = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  if (i >= M || gg >= NG) return;
  const int n = gr.count(gg);
  AccT comp[64];
  for (int p = 0; p < gr.lp1; ++p) comp[p] = X[i * ldx + gg * gr.lp1 + p];
  for (int t = 0; t < n; ++t) {
    AccT acc = 0;
    for (int p = 0; p < gr.lp1; ++p) acc += comp[p] * Cs[t * gr.lp1 + p];
    store(dA + i * ldda + gg * gr.L + t, acc);
  }
}

// dB[gg*L + t][j] = sum_p d[p,t] X[(g,p)][j]  (X: Kp x N, pitch ldx)
template <typename AccT, typename OutT>
__global__ void __launch_bounds__(256) expand_cols_kernel(const AccT* __restrict__ X, int64_t ldx, int64_t N,
                                                          Groups gr, const AccT* __restrict__ Ds,
                                                          OutT* __restrict__ dB, int64_t lddb) {
  const int64_t gg = blockIdx.x;
  const int64_t j = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int n = gr.count(gg);
  AccT comp[64];
  for (int p = 0; p < gr.lp1; ++p) comp[p] = X[(gg * gr.lp1 + p) * ldx + j];
  for (int t = 0; t < n; ++t) {
    AccT acc = 0;
    for (int p = 0; p < gr.lp1; ++p) acc += Ds[p * gr.L + t] * comp[p];
    store(dB + (gg * gr.L + t) * lddb + j, acc);
  }
}

// Y[i][j] = sum_k A(i,k) B(k,j) in double with general strides (correctness path).
__global__ void __launch_bounds__(256) gemm_f64_strided_kernel(const double* __restrict__ A, int64_t sam,
                                                               int64_t sak, const double* __restrict__ B,
                                                               int64_t sbk, int64_t sbn, double* __restrict__ Y,
                                                               int64_t ldy, int64_t M, int64_t N, int64_t K) {
  __shared__ double sA[32][33];
  __shared__ double sB[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int64_t i0 = static_cast<int64_t>(blockIdx.y) * 32, j0 = static_cast<int64_t>(blockIdx.x) * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
    for (int r = 0; r < 4; ++r) {
      const int row = ty + 8 * r;
      sA[row][tx] = (i0 + row < M && k0 + tx < K) ? A[(i0 + row) * sam + (k0 + tx) * sak] : 0.0;
      sB[row][tx] = (k0 + row < K && j0 + tx < N) ? B[(k0 + row) * sbk + (j0 + tx) * sbn] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < 32; ++kk) {
      const double b = sB[kk][tx];
      for (int r = 0; r < 4; ++r) acc[r] = fma(sA[ty + 8 * r][kk], b, acc[r]);
    }
    __syncthreads();
  }
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty + 8 * r, j = j0 + tx;
    if (i < M && j < N) Y[i * ldy + j] = acc[r];
  }
}

Groups groups_of(const GemmGeom& g) {
  Groups gr;
  gr.K = g.K;
  gr.L = g.L;
  gr.lp1 = g.lp1;
  return gr;
}

}  // namespace

cudaError_t launch_project_cols_nt_bf16(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g,
                                        const float* Ds, uint16_t* Bd, int64_t ldo, cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (NG == 0 || g.N == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(NG), static_cast<unsigned>(ceil_div(g.N, 256)));
  if (in_dtype == PJ_F32)
    project_cols_nt_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(B), ldb, g.N, groups_of(g), Ds,
                                                        Bd, ldo);
  else
    project_cols_nt_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(B), ldb, g.N,
                                                                groups_of(g), Ds, Bd, ldo);
  return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const void* X, int in_dtype, int64_t ldx, int64_t rows, int64_t cols,
                                  uint16_t* out, int64_t ldo, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(ceil_div(cols, 32)), static_cast<unsigned>(ceil_div(rows, 32)));
  if (in_dtype == PJ_F32)
    transpose_bf16_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(X), ldx, rows, cols, out, ldo);
  else
    transpose_bf16_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), ldx, rows,
                                                               cols, out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_convert_bf16(const void* X, int in_dtype, int64_t ldx, int64_t rows, int64_t cols, uint16_t* out,
                                int64_t ldo, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(rows), static_cast<unsigned>(ceil_div(cols, 256)));
  if (in_dtype == PJ_F32)
    convert_bf16_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(X), ldx, rows, cols, out, ldo);
  else
    convert_bf16_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), ldx, rows, cols,
                                                             out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_expand_rows(const void* X, int acc_dtype, int64_t ldx, const GemmGeom& g, const void* Cs,
                               void* dA, int out_dtype, int64_t ldda, cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (NG == 0 || g.M == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(g.M), static_cast<unsigned>(ceil_div(NG, 256)));
  if (acc_dtype == PJ_F64)
    expand_rows_kernel<double, double><<<grid, 256, 0, st>>>(static_cast<const double*>(X), ldx, g.M, groups_of(g),
                                                             NG, static_cast<const double*>(Cs),
                                                             static_cast<double*>(dA), ldda);
  else if (out_dtype == PJ_BF16)
    expand_rows_kernel<float, __nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.M,
                                                                   groups_of(g), NG, static_cast<const float*>(Cs),
                                                                   static_cast<__nv_bfloat16*>(dA), ldda);
  else
    expand_rows_kernel<float, float><<<grid, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.M, groups_of(g), NG,
                                                           static_cast<const float*>(Cs), static_cast<float*>(dA),
                                                           ldda);
  return cudaGetLastError();
}

cudaError_t launch_expand_cols(const void* X, int acc_dtype, int64_t ldx, const GemmGeom& g, const void* Ds,
                               void* dB, int out_dtype, int64_t lddb, cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (NG == 0 || g.N == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(NG), static_cast<unsigned>(ceil_div(g.N, 256)));
  if (acc_dtype == PJ_F64)
    expand_cols_kernel<double, double><<<grid, 256, 0, st>>>(static_cast<const double*>(X), ldx, g.N, groups_of(g),
                                                             static_cast<const double*>(Ds),
                                                             static_cast<double*>(dB), lddb);
  else if (out_dtype == PJ_BF16)
    expand_cols_kernel<float, __nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.N,
                                                                   groups_of(g), static_cast<const float*>(Ds),
                                                                   static_cast<__nv_bfloat16*>(dB), lddb);
  else
    expand_cols_kernel<float, float><<<grid, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.N, groups_of(g),
                                                           static_cast<const float*>(Ds), static_cast<float*>(dB),
                                                           lddb);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64_strided(const double* A, int64_t sam, int64_t sak, const double* B, int64_t sbk,
                                    int64_t sbn, double* Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                                    cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(ceil_div(N, 32)), static_cast<unsigned>(ceil_div(M, 32)));
  gemm_f64_strided_kernel<<<grid, 256, 0, st>>>(A, sam, sak, B, sbk, sbn, Y, ldy, M, N, K);
  return cudaGetLastError();
}

}  // namespace pj
