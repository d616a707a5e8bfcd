// Projection kernels (Sec. III-B): every group of L consecutive inner-dimension
// values of a row of A is multiplied by the kept columns of C, every group of
// a column of B by the kept rows of D (Fig. 5 and its description), and the
// CONV signal / templates are projected per group (Fig. 6, Eq. 11-12).
// These kernels stream HBM; the arithmetic is FP32 (FP64 for the double path).
#include <cuda_bf16.h>

#include "common.hpp"

namespace pj {
namespace {

__device__ __forceinline__ float load_as_float(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_as_float(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_value(uint16_t b) {
  return __bfloat162float(__ushort_as_bfloat16(b));
}

// Column of component (block b, projection p, group g) in the reduced inner
// dimension: blocks are laid out one after another, R components each (the
// last block may hold fewer), projection-major inside a block.
struct CompIndex {
  int64_t Kb, K, R;
  int L, lp1;
  __device__ __forceinline__ void locate(int64_t gg, int64_t& base, int64_t& G, int64_t& g) const {
    const int64_t GB = Kb / L;               // groups in a full block
    const int64_t b = gg / GB;
    g = gg - b * GB;
    const int64_t kb = K - b * Kb < Kb ? K - b * Kb : Kb;
    G = (kb + L - 1) / L;
    base = b * R;
  }
};

// ---- rows of A -> A_c (BF16, hi [+ lo]) ---------------------------------
// One thread per (row i, group gg); writes for fixed p are contiguous in g.
template <typename InT>
__global__ void __launch_bounds__(256) project_rows_bf16_kernel(const InT* __restrict__ A, int64_t lda, int64_t M,
                                                                CompIndex ci, int64_t NG, int64_t pitch,
                                                                int64_t Kp, int64_t Kp_pad, int nsplit,
                                                                const float* __restrict__ Cs,
                                                                uint16_t* __restrict__ Ac) {
  __shared__ float sC[64 * 64];
  for (int e = threadIdx.x; e < ci.L * ci.lp1; e += blockDim.x) sC[e] = Cs[e];
  __syncthreads();
  const int64_t i = blockIdx.x;
  const int64_t gg = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  uint16_t* out = Ac + i * pitch;
  if (gg == 0)
    for (int64_t c = Kp; c < Kp_pad; ++c)
      for (int s = 0; s < nsplit; ++s) out[s * Kp_pad + c] = 0;
  if (gg >= NG) return;
  const InT* a = A + i * lda + gg * ci.L;
  const int n = static_cast<int>(ci.K - gg * ci.L < ci.L ? ci.K - gg * ci.L : ci.L);
  float x[64];
#pragma unroll 8
  for (int t = 0; t < 64; ++t)
    if (t < ci.L) x[t] = t < n ? load_as_float(a + t) : 0.0f;
  int64_t base, G, g;
  ci.locate(gg, base, G, g);
  for (int p = 0; p < ci.lp1; ++p) {
    float acc = 0.0f;
#pragma unroll 8
    for (int t = 0; t < 64; ++t)
      if (t < ci.L) acc = fmaf(x[t], sC[t * ci.lp1 + p], acc);
    const int64_t col = base + p * G + g;
    const uint16_t hi = bf16_bits(acc);
    out[col] = hi;
    if (nsplit > 1) out[Kp_pad + col] = bf16_bits(acc - bf16_value(hi));
  }
}

// ---- columns of B -> B_d stored transposed (N x pitch, K-major) -----------
// A block stages 32 columns x TG groups of B in shared memory (coalesced
// along the columns), then each thread projects one (column, group) and
// writes its components; consecutive threads hold consecutive groups of the
// same column, so the writes of one projection are contiguous.
template <typename InT>
__global__ void __launch_bounds__(256) project_cols_bf16_kernel(const InT* __restrict__ B, int64_t ldb, int64_t N,
                                                                CompIndex ci, int64_t NG, int TG, int64_t pitch,
                                                                int64_t Kp, int64_t Kp_pad, int nsplit,
                                                                const float* __restrict__ Ds,
                                                                uint16_t* __restrict__ Bd) {
  extern __shared__ float smem[];
  float* sD = smem;                        // lp1 x L
  const int rowlen = TG * ci.L + 4;        // padded pitch of one staged column
  float* sB = smem + 64 * 64;              // 32 x rowlen
  const int L = ci.L;
  for (int e = threadIdx.x; e < ci.lp1 * L; e += blockDim.x) sD[e] = Ds[e];
  const int64_t j0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int64_t gg0 = static_cast<int64_t>(blockIdx.x) * TG;
  const int64_t k0 = gg0 * L;
  const int nk = TG * L;
  for (int e = threadIdx.x; e < nk * 32; e += blockDim.x) {
    const int kk = e / 32, jj = e % 32;
    const int64_t k = k0 + kk, j = j0 + jj;
    sB[jj * rowlen + kk] = (k < ci.K && j < N) ? load_as_float(B + k * ldb + j) : 0.0f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TG * 32; e += blockDim.x) {
    const int gl = e % TG, jj = e / TG;
    const int64_t gg = gg0 + gl, j = j0 + jj;
    if (gg >= NG || j >= N) continue;
    int64_t base, G, g;
    ci.locate(gg, base, G, g);
    const float* x = sB + jj * rowlen + gl * L;
    uint16_t* out = Bd + j * pitch;
    for (int p = 0; p < ci.lp1; ++p) {
      float acc = 0.0f;
      for (int t = 0; t < L; ++t) acc = fmaf(sD[p * L + t], x[t], acc);
      const int64_t col = base + p * G + g;
      const uint16_t hi = bf16_bits(acc);
      out[col] = hi;
      if (nsplit > 1) out[Kp_pad + col] = bf16_bits(acc - bf16_value(hi));
    }
  }
}

__global__ void zero_pad_cols_kernel(uint16_t* __restrict__ X, int64_t rows, int64_t pitch, int64_t Kp,
                                     int64_t Kp_pad, int nsplit) {
  const int64_t width = Kp_pad - Kp;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = rows * width * nsplit;
  if (e >= total) return;
  const int64_t c = e % width;
  const int64_t s = (e / width) % nsplit;
  const int64_t r = e / (width * nsplit);
  X[r * pitch + s * Kp_pad + Kp + c] = 0;
}

// ---- FP64 path ------------------------------------------------------------
__global__ void project_rows_f64_kernel(const double* __restrict__ A, int64_t lda, int64_t M, CompIndex ci,
                                        int64_t NG, int64_t Kp, const double* __restrict__ Cs,
                                        double* __restrict__ Ac) {
  const int64_t i = blockIdx.x;
  const int64_t gg = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  if (i >= M || gg >= NG) return;
  const double* a = A + i * lda + gg * ci.L;
  const int n = static_cast<int>(ci.K - gg * ci.L < ci.L ? ci.K - gg * ci.L : ci.L);
  int64_t base, G, g;
  ci.locate(gg, base, G, g);
  for (int p = 0; p < ci.lp1; ++p) {
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(a[t], Cs[t * ci.lp1 + p], acc);
    Ac[i * Kp + base + p * G + g] = acc;
  }
}

__global__ void project_cols_f64_kernel(const double* __restrict__ B, int64_t ldb, int64_t N, CompIndex ci,
                                        int64_t NG, const double* __restrict__ Ds, double* __restrict__ Bd) {
  const int64_t j = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  const int64_t gg = blockIdx.x;
  if (j >= N || gg >= NG) return;
  const int n = static_cast<int>(ci.K - gg * ci.L < ci.L ? ci.K - gg * ci.L : ci.L);
  int64_t base, G, g;
  ci.locate(gg, base, G, g);
  for (int p = 0; p < ci.lp1; ++p) {
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(Ds[p * ci.L + t], B[(gg * ci.L + t) * ldb + j], acc);
    Bd[(base + p * G + g) * N + j] = acc;
  }
}

// ---- CONV: signal and templates -------------------------------------------
// Box-basis form of the Haar projection with l+1 a power of two: the kept
// span is the functions constant on aligned runs of Lb = T / R samples, with
// orthonormal basis 1/sqrt(Lb) on each run.  The projected signal at
// position x is b[x] = sum_{u < Lb} s[x + u] / sqrt(Lb).  It is stored phase-
// split, with eight element shifts so every row view starts 16-byte aligned:
//   G[(sigma * Lb + phi) * P + y] = b[phi + Lb * (y + sigma)]  (0 where b is undefined).
// One thread per (phi, Y) computes b[phi + Lb * Y] once and writes it to the
// eight shifted copies (y = Y - sigma).
__global__ void __launch_bounds__(256) conv_signal_kernel(const float* __restrict__ s, int64_t S, int Lb, int64_t P,
                                                          float scale, uint16_t* __restrict__ G) {
  const int64_t Y = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int phi = blockIdx.y;
  if (Y >= P + 7) return;
  const int64_t x = phi + static_cast<int64_t>(Lb) * Y;
  float v = 0.0f;
  if (x + Lb <= S) {
    for (int u = 0; u < Lb; ++u) v += __ldg(s + x + u);
    v *= scale;
  }
  const uint16_t bits = bf16_bits(v);
#pragma unroll
  for (int sigma = 0; sigma < 8; ++sigma) {
    const int64_t y = Y - sigma;
    if (y >= 0 && y < P) G[(static_cast<int64_t>(sigma) * Lb + phi) * P + y] = bits;
  }
}

// Template pairs for the lag-paired reduced correlation: chunk c holds 128 rows
// of 64 components; row e*64 + t is template t's components [64(c-e), 64(c-e)+64)
// (zero outside [0, R) and for t >= nt).  Component g of template t is
// sum_{u < Lb} k_t[g*Lb + u] / sqrt(Lb).
__global__ void __launch_bounds__(256) conv_templates_kernel(const float* __restrict__ k, int64_t T, int64_t nt,
                                                             int Lb, int Kc, float scale,
                                                             uint16_t* __restrict__ TP) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t total = static_cast<int64_t>(Kc + 1) * 128 * 64;
  if (e >= total) return;
  const int i = static_cast<int>(e % 64);
  const int row = static_cast<int>((e / 64) % 128);
  const int c = static_cast<int>(e / (64 * 128));
  const int ee = row / 64, t = row % 64;
  const int cc = c - ee;
  float v = 0.0f;
  if (t < nt && cc >= 0 && cc < Kc) {
    const int64_t g = static_cast<int64_t>(cc) * 64 + i;
    const float* kt = k + t * T + g * Lb;
    for (int u = 0; u < Lb; ++u) v += __ldg(kt + u);
    v *= scale;
  }
  TP[e] = bf16_bits(v);
}

}  // namespace

static CompIndex comp_index(const GemmGeom& g) {
  CompIndex ci;
  ci.Kb = g.Kb;
  ci.K = g.K;
  ci.R = g.R;
  ci.L = g.L;
  ci.lp1 = g.lp1;
  return ci;
}

cudaError_t launch_project_rows_bf16(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs,
                                     uint16_t* Ac, cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  const int64_t pitch = g.Kp_pad * g.nsplit;
  if (g.M == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(g.M), static_cast<unsigned>(ceil_div(NG > 0 ? NG : 1, 256)));
  if (in_dtype == PJ_F32)
    project_rows_bf16_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, g.M, comp_index(g),
                                                          NG, pitch, g.Kp, g.Kp_pad, g.nsplit, Cs, Ac);
  else
    project_rows_bf16_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(A), lda, g.M,
                                                                  comp_index(g), NG, pitch, g.Kp, g.Kp_pad,
                                                                  g.nsplit, Cs, Ac);
  return cudaGetLastError();
}

cudaError_t launch_project_cols_bf16(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds,
                                     uint16_t* Bd, cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  const int64_t pitch = g.Kp_pad * g.nsplit;
  if (g.N == 0) return cudaSuccess;
  const int TG = g.L <= 8 ? 32 : 256 / g.L;
  const size_t smem = (64 * 64 + 32 * (TG * g.L + 4)) * sizeof(float);
  dim3 grid(static_cast<unsigned>(ceil_div(NG > 0 ? NG : 1, TG)), static_cast<unsigned>(ceil_div(g.N, 32)));
  cudaError_t e;
  if (in_dtype == PJ_F32) {
    e = cudaFuncSetAttribute(project_cols_bf16_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    project_cols_bf16_kernel<float><<<grid, 256, smem, st>>>(static_cast<const float*>(B), ldb, g.N, comp_index(g),
                                                             NG, TG, pitch, g.Kp, g.Kp_pad, g.nsplit, Ds, Bd);
  } else {
    e = cudaFuncSetAttribute(project_cols_bf16_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    project_cols_bf16_kernel<__nv_bfloat16><<<grid, 256, smem, st>>>(static_cast<const __nv_bfloat16*>(B), ldb,
                                                                     g.N, comp_index(g), NG, TG, pitch, g.Kp,
                                                                     g.Kp_pad, g.nsplit, Ds, Bd);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (g.Kp_pad > g.Kp) {
    const int64_t total = g.N * (g.Kp_pad - g.Kp) * g.nsplit;
    zero_pad_cols_kernel<<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(Bd, g.N, pitch, g.Kp,
                                                                                       g.Kp_pad, g.nsplit);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_project_rows_f64(const double* A, int64_t lda, const GemmGeom& g, const double* Cs, double* Ac,
                                    cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (g.M == 0 || NG == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(g.M), static_cast<unsigned>(ceil_div(NG, 128)));
  project_rows_f64_kernel<<<grid, 128, 0, st>>>(A, lda, g.M, comp_index(g), NG, g.Kp, Cs, Ac);
  return cudaGetLastError();
}

cudaError_t launch_project_cols_f64(const double* B, int64_t ldb, const GemmGeom& g, const double* Ds, double* Bd,
                                    cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (g.N == 0 || NG == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(NG), static_cast<unsigned>(ceil_div(g.N, 128)));
  project_cols_f64_kernel<<<grid, 128, 0, st>>>(B, ldb, g.N, comp_index(g), NG, Ds, Bd);
  return cudaGetLastError();
}

cudaError_t launch_conv_project_signal(const float* s, const ConvGeom& g, uint16_t* G, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>(ceil_div(g.P + 7, 256)), static_cast<unsigned>(g.Lb));
  conv_signal_kernel<<<grid, 256, 0, st>>>(s, g.S, g.Lb, g.P, 1.0f / sqrtf(static_cast<float>(g.Lb)), G);
  return cudaGetLastError();
}

cudaError_t launch_conv_project_templates(const float* k, const ConvGeom& g, uint16_t* TP, cudaStream_t st) {
  const int64_t total = static_cast<int64_t>(g.Kc + 1) * 128 * 64;
  conv_templates_kernel<<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(
      k, g.T, g.nt, g.Lb, g.Kc, 1.0f / sqrtf(static_cast<float>(g.Lb)), TP);
  return cudaGetLastError();
}

}  // namespace pj
