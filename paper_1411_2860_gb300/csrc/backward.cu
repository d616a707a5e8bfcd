// Kernels of the projected-GEMM gradients.  With Y = A P B and
// P = blockdiag(C_R D_R) (Sec. III-B; Eq. 15 truncated as in Eq. 8):
//   dA = dY (P B)^T = expand_C(dY B_d^T),   dB = (A P)^T dY = expand_D(A_c^T dY)
// where B_d, A_c are the projected operands (recomputed, not stored) and the
// expansions map components back to samples:
//   expand_C(X)[i][gL+t] = sum_p X[i][(g,p)] c[t,p],
//   expand_D(X)[gL+t][j] = sum_p d[p,t] X[(g,p)][j].
// The two reduced products run on the tcgen05 GEMM (BF16) or the FP64 kernel;
// in the BF16 path with L = 8 and l+1 a power of two the GEMM epilogue does the
// expansion itself (gemm_tc.cu), and the kernels here serve the other cases.
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

// ---- 16-byte paths for the BF16 backward (L = 8, aligned rows) -----------

__device__ __forceinline__ uint16_t bf16u(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t pk2(uint16_t a, uint16_t b) { return a | (uint32_t(b) << 16); }
__device__ __forceinline__ uint4 pk8(const uint16_t (&v)[8]) {
  return make_uint4(pk2(v[0], v[1]), pk2(v[2], v[3]), pk2(v[4], v[5]), pk2(v[6], v[7]));
}

// Eight consecutive values (16-byte aligned) as BF16 bits.
__device__ __forceinline__ void load8_bf16(const float* p, uint16_t (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = bf16u(a.x); v[1] = bf16u(a.y); v[2] = bf16u(a.z); v[3] = bf16u(a.w);
  v[4] = bf16u(b.x); v[5] = bf16u(b.y); v[6] = bf16u(b.z); v[7] = bf16u(b.w);
}
__device__ __forceinline__ void load8_bf16(const __nv_bfloat16* p, uint16_t (&v)[8]) {
  const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = static_cast<uint16_t>(w[k] & 0xffffu);
    v[2 * k + 1] = static_cast<uint16_t>(w[k] >> 16);
  }
}
__device__ __forceinline__ void load8_float(const float* p, float (&x)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void load8_float(const __nv_bfloat16* p, float (&x)[8]) {
  uint16_t v[8];
  load8_bf16(p, v);
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = __uint_as_float(uint32_t(v[k]) << 16);
}


// X (rows x cols, pitch ldx) -> BF16 copy (pitch ldo), eight values per thread.
template <typename InT>
__global__ void __launch_bounds__(256) convert8_kernel(const InT* __restrict__ X, int64_t ldx, int64_t rows,
                                                       int64_t cols, uint16_t* __restrict__ out, int64_t ldo) {
  const int64_t c8 = (cols + 7) / 8;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * c8) return;
  const int64_t r = e / c8, c = (e - r * c8) * 8;
  uint16_t v[8];
  if (c + 8 <= cols) {
    load8_bf16(X + r * ldx + c, v);
    *reinterpret_cast<uint4*>(out + r * ldo + c) = pk8(v);
  } else {
    for (int64_t j = c; j < cols; ++j) out[r * ldo + j] = bf16u(to_float(X[r * ldx + j]));
  }
}

// dA[i][8 gg + t] = sum_p X[i][gg (l+1) + p] c[t,p]  (L = 8), one thread per
// (i, four consecutive groups): 4 (l+1) contiguous reads, 4 x 8 contiguous writes.
template <typename OutT>
__global__ void __launch_bounds__(256) expand_rows8_kernel(const float* __restrict__ X, int64_t ldx, int64_t M,
                                                           int64_t K, int lp1, int64_t NG,
                                                           const float* __restrict__ Cs, OutT* __restrict__ dA,
                                                           int64_t ldda) {
  __shared__ float sC[64];
  if (threadIdx.x < 8 * lp1) sC[threadIdx.x] = Cs[threadIdx.x];
  __syncthreads();
  const int64_t NQ = (NG + 3) / 4;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M * NQ) return;
  const int64_t i = e / NQ, g0 = (e - i * NQ) * 4;
  const float* xr = X + i * ldx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t gg = g0 + q;
    if (gg >= NG) break;
    float comp[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) comp[p] = p < lp1 ? __ldg(xr + gg * lp1 + p) : 0.0f;
    float y[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float acc = 0.0f;
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if (p < lp1) acc = fmaf(comp[p], sC[t * lp1 + p], acc);
      y[t] = acc;
    }
    OutT* o = dA + i * ldda + gg * 8;
    const int n = static_cast<int>(K - gg * 8 < 8 ? K - gg * 8 : 8);
    if (n == 8) {
      if (sizeof(OutT) == 2) {
        uint16_t v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = bf16u(y[t]);
        *reinterpret_cast<uint4*>(o) = pk8(v);
      } else {
        reinterpret_cast<float4*>(o)[0] = make_float4(y[0], y[1], y[2], y[3]);
        reinterpret_cast<float4*>(o)[1] = make_float4(y[4], y[5], y[6], y[7]);
      }
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < n) store(o + t, y[t]);
    }
  }
}

// dB[8 gg + t][j .. j+3] = sum_p d[p,t] X[gg (l+1) + p][j .. j+3]  (L = 8), one
// thread per (gg, four columns).
template <typename OutT>
__global__ void __launch_bounds__(256) expand_cols8_kernel(const float* __restrict__ X, int64_t ldx, int64_t N,
                                                           int64_t K, int lp1, int64_t NG,
                                                           const float* __restrict__ Ds, OutT* __restrict__ dB,
                                                           int64_t lddb) {
  __shared__ float sD[64];
  if (threadIdx.x < 8 * lp1) sD[threadIdx.x] = Ds[threadIdx.x];
  __syncthreads();
  const int64_t nq = (N + 3) / 4;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= NG * nq) return;
  const int64_t gg = e / nq, j = (e - gg * nq) * 4;
  const int nj = static_cast<int>(N - j < 4 ? N - j : 4);
  float4 comp[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    comp[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (p < lp1) {
      const float* xr = X + (gg * lp1 + p) * ldx + j;
      if (nj == 4) {
        comp[p] = __ldg(reinterpret_cast<const float4*>(xr));
      } else {
        comp[p].x = xr[0];
        if (nj > 1) comp[p].y = xr[1];
        if (nj > 2) comp[p].z = xr[2];
      }
    }
  }
  const int n = static_cast<int>(K - gg * 8 < 8 ? K - gg * 8 : 8);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t >= n) break;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      if (p < lp1) {
        const float d = sD[p * 8 + t];
        acc.x = fmaf(d, comp[p].x, acc.x);
        acc.y = fmaf(d, comp[p].y, acc.y);
        acc.z = fmaf(d, comp[p].z, acc.z);
        acc.w = fmaf(d, comp[p].w, acc.w);
      }
    }
    OutT* o = dB + (gg * 8 + t) * lddb + j;
    if (nj == 4) {
      if (sizeof(OutT) == 2)
        *reinterpret_cast<uint2*>(o) = make_uint2(pk2(bf16u(acc.x), bf16u(acc.y)), pk2(bf16u(acc.z), bf16u(acc.w)));
      else
        *reinterpret_cast<float4*>(o) = acc;
    } else {
      const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
      for (int q = 0; q < nj; ++q) store(o + q, a4[q]);
    }
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

static bool rows16(const void* p, int64_t ld, size_t es) {
  return reinterpret_cast<uintptr_t>(p) % 16 == 0 && (ld * static_cast<int64_t>(es)) % 16 == 0;
}

cudaError_t launch_convert_bf16(const void* X, int in_dtype, int64_t ldx, int64_t rows, int64_t cols, uint16_t* out,
                                int64_t ldo, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  const size_t es = in_dtype == PJ_F32 ? 4 : 2;
  if (rows16(X, ldx, es) && rows16(out, ldo, 2)) {
    const unsigned blocks = static_cast<unsigned>(ceil_div(rows * ceil_div(cols, 8), 256));
    if (in_dtype == PJ_F32)
      convert8_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), ldx, rows, cols, out, ldo);
    else
      convert8_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), ldx, rows, cols,
                                                             out, ldo);
    return cudaGetLastError();
  }
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
  const size_t oes = out_dtype == PJ_BF16 ? 2 : 4;
  if (acc_dtype == PJ_F32 && g.L == 8 && rows16(dA, ldda, oes)) {
    const unsigned blocks = static_cast<unsigned>(ceil_div(g.M * ceil_div(NG, 4), 256));
    if (out_dtype == PJ_BF16)
      expand_rows8_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.M, g.K, g.lp1,
                                                                 NG, static_cast<const float*>(Cs),
                                                                 static_cast<__nv_bfloat16*>(dA), ldda);
    else
      expand_rows8_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.M, g.K, g.lp1, NG,
                                                         static_cast<const float*>(Cs), static_cast<float*>(dA), ldda);
    return cudaGetLastError();
  }
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
  const size_t oes = out_dtype == PJ_BF16 ? 2 : 4;
  // 8-byte (BF16) or 16-byte (FP32) stores of four columns; 16-byte loads of X rows.
  if (acc_dtype == PJ_F32 && g.L == 8 && rows16(X, ldx, 4) && reinterpret_cast<uintptr_t>(dB) % 16 == 0 &&
      (lddb * static_cast<int64_t>(oes)) % (4 * oes) == 0) {
    const unsigned blocks = static_cast<unsigned>(ceil_div(NG * ceil_div(g.N, 4), 256));
    if (out_dtype == PJ_BF16)
      expand_cols8_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.N, g.K, g.lp1,
                                                                 NG, static_cast<const float*>(Ds),
                                                                 static_cast<__nv_bfloat16*>(dB), lddb);
    else
      expand_cols8_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), ldx, g.N, g.K, g.lp1, NG,
                                                         static_cast<const float*>(Ds), static_cast<float*>(dB), lddb);
    return cudaGetLastError();
  }
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
