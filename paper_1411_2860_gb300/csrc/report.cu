// A-posteriori report of a projected product: algorithmic work, and bounds on
// its two errors computed from the inputs (Sec. III-A: the truncation of Eq. 8
// per block; the rounding of the reduced product).
//
// Truncation.  Y - Y_R = sum_b A_b (I - P_b) B_b over the blocks b of the inner
// dimension, P_b the projector onto the kept projections of each group.  For an
// orthonormal basis P_b is symmetric and idempotent, so Cauchy-Schwarz per block
// gives ||Y - Y_R||_F <= sum_b ||A_b (I - P_b)||_F ||(I - P_b) B_b||_F, and by
// Parseval ||A_b (I - P_b)||_F^2 = ||A_b||_F^2 - ||A_b C_R||_F^2 (likewise for B).
// One pass over A and B computes the three sums per block in double.
//
// Rounding.  Every output obeys |y - y_R| <= f * sum_k |a|_k |b|_k with the
// component bounds |a|_k = sum_t |A_t| |C_tp| (the forward bound of the kernels'
// arithmetic), so ||Y - Y_R||_F <= f * ||(|A| |C|)||_F * ||(|D| |B|)||_F.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.hpp"

namespace pj {
namespace {

__device__ __forceinline__ double ld_input(const float* p) { return static_cast<double>(__ldg(p)); }
__device__ __forceinline__ double ld_input(const double* p) { return __ldg(p); }
__device__ __forceinline__ double ld_input(const __nv_bfloat16* p) {
  return static_cast<double>(__bfloat162float(*p));
}

// Rows of A: warp w takes (row i, block b) = (w / nb, w % nb); its lanes take the
// block's groups in turn.  acc[3 b + 0..2] += sum A^2, sum (A C)^2, sum (|A| |C|)^2.
template <typename InT>
__global__ void __launch_bounds__(256) report_rows_kernel(const InT* __restrict__ A, int64_t lda, int64_t M, int64_t K,
                                                          int64_t Kb, int L, int lp1, const double* __restrict__ Cs,
                                                          int64_t nb, double* acc) {
  const int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (w >= M * nb) return;  // the same for the whole warp
  const int64_t i = w / nb, b = w - i * nb;
  const int64_t k0 = b * Kb, k1 = k0 + Kb < K ? k0 + Kb : K;
  const int64_t groups = (k1 - k0 + L - 1) / L;
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t g = lane; g < groups; g += 32) {
    double x[kMaxL];
    for (int t = 0; t < L; ++t) {
      const int64_t k = k0 + g * L + t;
      x[t] = k < k1 ? ld_input(A + i * lda + k) : 0.0;
      s[0] += x[t] * x[t];
    }
    for (int p = 0; p < lp1; ++p) {
      double v = 0.0, va = 0.0;
      for (int t = 0; t < L; ++t) {
        v = fma(x[t], Cs[t * lp1 + p], v);
        va = fma(fabs(x[t]), fabs(Cs[t * lp1 + p]), va);
      }
      s[1] += v * v;
      s[2] += va * va;
    }
  }
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
  if (lane == 0)
    for (int q = 0; q < 3; ++q) atomicAdd(acc + 3 * b + q, s[q]);
}

// Columns of B: thread (j, b) with j fastest, so the reads of one row of B are
// coalesced.  acc[3 b + 0..2] += sum B^2, sum (D B)^2, sum (|D| |B|)^2.
template <typename InT>
__global__ void __launch_bounds__(256) report_cols_kernel(const InT* __restrict__ B, int64_t ldb, int64_t N, int64_t K,
                                                          int64_t Kb, int L, int lp1, const double* __restrict__ Ds,
                                                          int64_t nb, double* acc) {
  const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (u >= N * nb) return;
  const int64_t b = u / N, j = u - b * N;
  const int64_t k0 = b * Kb, k1 = k0 + Kb < K ? k0 + Kb : K;
  const int64_t groups = (k1 - k0 + L - 1) / L;
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t g = 0; g < groups; ++g) {
    double x[kMaxL];
    for (int t = 0; t < L; ++t) {
      const int64_t k = k0 + g * L + t;
      x[t] = k < k1 ? ld_input(B + k * ldb + j) : 0.0;
      s[0] += x[t] * x[t];
    }
    for (int p = 0; p < lp1; ++p) {
      double v = 0.0, va = 0.0;
      for (int t = 0; t < L; ++t) {
        v = fma(Ds[p * L + t], x[t], v);
        va = fma(fabs(Ds[p * L + t]), fabs(x[t]), va);
      }
      s[1] += v * v;
      s[2] += va * va;
    }
  }
  for (int q = 0; q < 3; ++q) atomicAdd(acc + 3 * b + q, s[q]);
}

template <typename InT>
cudaError_t launch_report(const void* A, int64_t lda, const void* B, int64_t ldb, const GemmGeom& g, const double* Cs,
                          const double* Ds, int64_t nb, double* accA, double* accB, cudaStream_t st) {
  if (g.M > 0) {
    const int64_t threads = g.M * nb * 32;
    report_rows_kernel<InT><<<static_cast<unsigned>(ceil_div(threads, 256)), 256, 0, st>>>(
        static_cast<const InT*>(A), lda, g.M, g.K, g.Kb, g.L, g.lp1, Cs, nb, accA);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (g.N > 0) {
    const int64_t threads = g.N * nb;
    report_cols_kernel<InT><<<static_cast<unsigned>(ceil_div(threads, 256)), 256, 0, st>>>(
        static_cast<const InT*>(B), ldb, g.N, g.K, g.Kb, g.L, g.lp1, Ds, nb, accB);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

size_t report_ws_bytes(int64_t nb) { return align_up(kHeaderBytes + kBasisBytes) + align_up(sizeof(double) * 6 * nb); }

double gamma_n(double n, double u) { return n * u / (1.0 - n * u); }

}  // namespace
}  // namespace pj

using namespace pj;

extern "C" {

size_t proj_gemm_report_workspace_size(int64_t K, int64_t block_k) {
  if (K < 0 || block_k < 1) return 0;
  return report_ws_bytes(K > 0 ? ceil_div(K, block_k) : 1);
}

pj_status proj_gemm_report(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                           int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                           const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream, pj_report* rep) {
  if (!rep) return fail(PJ_EINVAL, "report is NULL");
  if (!basis || !prec) return fail(PJ_EINVAL, "basis and precision must be non-NULL");
  GemmGeom g{};
  PJ_TRY(gemm_geom(M, N, K, block_k, R, basis, prec, &g));
  if (g.tier) return fail(PJ_EUNSUPPORTED, "proj_gemm_report does not cover an FP8 tier");
  if ((M > 0 && !A) || (N > 0 && !B)) return fail(PJ_EINVAL, "A and B must be non-NULL");
  if (in_dtype != PJ_F32 && in_dtype != PJ_BF16 && in_dtype != PJ_F64)
    return fail(PJ_EUNSUPPORTED, "in_dtype %d", in_dtype);
  if (out_dtype != PJ_F32 && out_dtype != PJ_BF16 && out_dtype != PJ_F64)
    return fail(PJ_EUNSUPPORTED, "out_dtype %d", out_dtype);
  if ((M > 0 && lda < K) || (N > 0 && ldb < N)) return fail(PJ_EINVAL, "lda >= K and ldb >= N required");
  const int64_t nb = K > 0 ? ceil_div(K, block_k) : 0;
  PJ_TRY(check_ws(workspace, ws_bytes, report_ws_bytes(nb > 0 ? nb : 1)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  PJ_TRY(stage_basis(basis, g.lp1, workspace, st));
  const BasisDev bd = basis_area(workspace);
  double* acc = reinterpret_cast<double*>(static_cast<char*>(workspace) + align_up(kHeaderBytes + kBasisBytes));
  std::vector<double> h(6 * (nb > 0 ? nb : 1), 0.0);
  if (nb > 0) {
    PJ_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 6 * nb, st));
    cudaError_t e = in_dtype == PJ_F64 ? launch_report<double>(A, lda, B, ldb, g, bd.Cs64, bd.Ds64, nb, acc, acc + 3 * nb, st)
                    : in_dtype == PJ_BF16 ? launch_report<__nv_bfloat16>(A, lda, B, ldb, g, bd.Cs64, bd.Ds64, nb, acc,
                                                                         acc + 3 * nb, st)
                                          : launch_report<float>(A, lda, B, ldb, g, bd.Cs64, bd.Ds64, nb, acc, acc + 3 * nb, st);
    PJ_CUDA_TRY(e);
    PJ_CUDA_TRY(cudaMemcpyAsync(h.data(), acc, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, st));
  }
  PJ_CUDA_TRY(cudaStreamSynchronize(st));
  int code = 0;
  PJ_CUDA_TRY(cudaMemcpy(&code, workspace, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) return fail(PJ_EINVAL, "the basis was rejected on the device (singular user matrix)");

  const double* hA = h.data();
  const double* hB = h.data() + 3 * nb;
  double nA = 0, nB = 0, cA = 0, cB = 0, trunc = 0;
  for (int64_t b = 0; b < nb; ++b) {
    nA += hA[3 * b];
    nB += hB[3 * b];
    cA += hA[3 * b + 2];
    cB += hB[3 * b + 2];
    // Parseval residuals; the slack covers the double rounding of the sums
    const double rA = hA[3 * b] - hA[3 * b + 1] + 1e-12 * hA[3 * b];
    const double rB = hB[3 * b] - hB[3 * b + 1] + 1e-12 * hB[3 * b];
    trunc += std::sqrt(rA > 0 ? rA : 0.0) * std::sqrt(rB > 0 ? rB : 0.0);
  }
  rep->norm_A = std::sqrt(nA);
  rep->norm_B = std::sqrt(nB);
  rep->trunc_bound = basis->kind == PJ_BASIS_USER ? -1.0 : trunc;
  // rounding factor of the kernels' arithmetic (components rounded with unit u,
  // projections summed over L terms and the reduced products over K' terms)
  const int passes = g.nsplit > 1 && g.compute != PJ_E4M3 ? 3 : 1;
  const double Kred = gemm_tiered(g) ? static_cast<double>(g.Kp + 2 * g.Kt) : static_cast<double>(g.Kp) * passes;
  double f = -1.0;
  if (g.compute == PJ_F64) {
    const double u = std::ldexp(1.0, -53);
    f = 2 * u + u * u + 2 * gamma_n(g.L, u) * (1 + u) * (1 + u) + 2 * gamma_n(Kred, u) * (1 + u) * (1 + u);
  } else if (g.compute == PJ_BF16) {
    const double u = std::ldexp(1.0, -8), u32 = std::ldexp(1.0, -24);
    // a tiered split keeps the plain term on its other projections: take the larger one
    const double lead = g.nsplit > 1 && !gemm_tiered(g) ? 4 * u * u : 2 * u + u * u;
    f = lead + 2 * gamma_n(g.L, u32) * (1 + u) * (1 + u) + 2 * gamma_n(Kred, u32) * (1 + u) * (1 + u);
  }
  rep->round_bound = f < 0 ? -1.0 : f * std::sqrt(cA) * std::sqrt(cB);
  const double es_in = in_dtype == PJ_F64 ? 8 : in_dtype == PJ_BF16 ? 2 : 4;
  const double es_out = out_dtype == PJ_F64 ? 8 : out_dtype == PJ_BF16 ? 2 : 4;
  const int nprod = g.compute == PJ_E4M3 ? (g.qsplit > 1 ? 3 : 1) : passes;
  const double Kprod = gemm_tiered(g) ? static_cast<double>(g.Kp + 2 * g.Kt) : static_cast<double>(g.Kp) * nprod;
  rep->alg_flops = 2.0 * M * N * Kprod + 2.0 * (static_cast<double>(M) + N) * K * g.lp1;
  rep->alg_bytes = es_in * (static_cast<double>(M) * K + static_cast<double>(K) * N) + es_out * M * N;
  return PJ_OK;
}

}  // extern "C"
