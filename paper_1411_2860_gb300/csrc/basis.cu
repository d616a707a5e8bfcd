// Projection basis builder (Sec. III-A, Eq. 5-7): builds C and D = C^-1 in FP64
// on the GPU, then the kept tables (lp1 consecutive columns of C and rows of D
// from projection p0 on: the first l+1 for the kept projections, p0 = 0; the
// next ones for an FP8 tier of truncated projections) in FP64 and FP32 for the
// projection kernels.
#include "common.hpp"
#include "tc.cuh"

namespace pj {
namespace {

constexpr int kBasisThreads = 256;

// Haar analysis vector j (j >= 1) at sample i: level = floor(log2 j), the
// wavelet's support has width L >> level and starts at (j - 2^level) * width;
// +1 on the first half of the support, -1 on the second half.
__device__ double haar_raw(int L, int i, int j) {
  if (j == 0) return 1.0;
  const int level = 31 - __clz(j);
  const int width = L >> level;
  const int start = (j - (1 << level)) * width;
  if (i < start || i >= start + width) return 0.0;
  return i < start + width / 2 ? 1.0 : -1.0;
}

__global__ void __launch_bounds__(kBasisThreads) basis_kernel(int kind, int L, int lp1, int p0, BasisDev b,
                                                               int* err) {
  __shared__ int s_fail;
  __shared__ int s_piv;
  const int tid = threadIdx.x, nth = blockDim.x;
  double* C = b.C64;
  double* D = b.D64;
  if (tid == 0) s_fail = 0;
  if (kind == PJ_BASIS_DCT2 || kind == PJ_BASIS_HAAR) {
    // Unit-length columns: the truncated product does not depend on column
    // scaling, and with orthogonal columns it makes D = C^T.  The squared
    // column norms have closed forms: DCT-II column j sums cos^2 over L
    // samples, L for j = 0 and L/2 otherwise; a Haar column is +-1 on its
    // support of width L >> floor(log2 j) (L for j = 0).  One pass, with no
    // read-back of the tables, so the kernel costs one trip to memory.
    for (int e = tid; e < L * L; e += nth) {
      const int i = e / L, j = e % L;
      double v;
      if (kind == PJ_BASIS_DCT2) {
        // cos(pi (i + 1/2) j / L) as cospi of the exact ratio (2i+1) j / (2L):
        // no multiplication by pi and no large-argument reduction
        v = cospi(static_cast<double>((2 * i + 1) * j) / (2 * L)) *
            (j == 0 ? rsqrt(static_cast<double>(L)) : sqrt(2.0 / L));
      } else {
        const int width = j == 0 ? L : (L >> (31 - __clz(j)));
        v = haar_raw(L, i, j) * rsqrt(static_cast<double>(width));
      }
      C[e] = v;
      D[j * L + i] = v;
      if (j >= p0 && j < p0 + lp1) {
        const int q = j - p0;
        b.Cs64[i * lp1 + q] = v;
        b.Cs32[i * lp1 + q] = static_cast<float>(v);
        b.CsT32[q * L + i] = static_cast<float>(v);
        b.Ds64[q * L + i] = v;
        b.Ds32[q * L + i] = static_cast<float>(v);
      }
    }
    return;
  } else {
    // User matrix: C = U, D = U^-1 by Gauss-Jordan with partial pivoting on
    // the augmented pair [W | D] (W starts as U, D as the identity).
    double* W = b.U64;
    double scale = 0.0;
    for (int e = tid; e < L * L; e += nth) {
      C[e] = W[e];
      D[e] = (e / L == e % L) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int e = 0; e < L * L; ++e) scale = fmax(scale, fabs(C[e]));
    for (int col = 0; col < L; ++col) {
      if (tid == 0) {
        int piv = col;
        for (int r = col + 1; r < L; ++r)
          if (fabs(W[r * L + col]) > fabs(W[piv * L + col])) piv = r;
        s_piv = piv;
        if (!(fabs(W[piv * L + col]) > 1e-13 * scale)) s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      const int piv = s_piv;
      if (piv != col)
        for (int j = tid; j < L; j += nth) {
          double t = W[col * L + j];
          W[col * L + j] = W[piv * L + j];
          W[piv * L + j] = t;
          t = D[col * L + j];
          D[col * L + j] = D[piv * L + j];
          D[piv * L + j] = t;
        }
      __syncthreads();
      const double inv = 1.0 / W[col * L + col];
      __syncthreads();
      for (int j = tid; j < L; j += nth) {
        W[col * L + j] *= inv;
        D[col * L + j] *= inv;
      }
      __syncthreads();
      for (int r = tid; r < L; r += nth) {
        if (r == col) continue;
        const double f = W[r * L + col];
        if (f == 0.0) continue;
        for (int j = 0; j < L; ++j) {
          W[r * L + j] -= f * W[col * L + j];
          D[r * L + j] -= f * D[col * L + j];
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_fail) {
      if (tid == 0) atomicCAS(err, 0, DEV_BAD_ARG);
      return;
    }
  }
  __syncthreads();
  for (int e = tid; e < L * lp1; e += nth) {
    const int i = e / lp1, p = e % lp1;
    b.Cs64[e] = C[i * L + p0 + p];
    b.Cs32[e] = static_cast<float>(C[i * L + p0 + p]);
    b.CsT32[p * L + i] = static_cast<float>(C[i * L + p0 + p]);
  }
  for (int e = tid; e < lp1 * L; e += nth) {
    b.Ds64[e] = D[p0 * L + e];
    b.Ds32[e] = static_cast<float>(D[p0 * L + e]);
  }
}

}  // namespace

cudaError_t launch_basis_build(int kind, int L, int lp1, BasisDev b, int* err, cudaStream_t st, int p0) {
  basis_kernel<<<1, kBasisThreads, 0, st>>>(kind, L, lp1, p0, b, err);
  return cudaGetLastError();
}

}  // namespace pj
