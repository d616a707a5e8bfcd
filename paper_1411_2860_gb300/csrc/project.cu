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

// Component order.  Every group of L consecutive inner-dimension values is
// projected on its own (the block-diagonal C_N, D_N of Eq. 15; the top-level
// block is a multiple of L, so no group straddles two blocks), and component
// p of global group gg sits at column gg * (l+1) + p of the reduced inner
// dimension.  A short last group (K not a multiple of L) is zero-extended.

// Widest aligned stores for a run of n BF16 values starting at dst, where dst
// is aligned to 2 * n bytes for n a power of two (n <= 16).
__device__ __forceinline__ void store_run(uint16_t* dst, const uint16_t* v, int n) {
  if (n == 8) {
    uint4 q;
    q.x = v[0] | (uint32_t(v[1]) << 16);
    q.y = v[2] | (uint32_t(v[3]) << 16);
    q.z = v[4] | (uint32_t(v[5]) << 16);
    q.w = v[6] | (uint32_t(v[7]) << 16);
    *reinterpret_cast<uint4*>(dst) = q;
  } else if (n == 4) {
    uint2 q;
    q.x = v[0] | (uint32_t(v[1]) << 16);
    q.y = v[2] | (uint32_t(v[3]) << 16);
    *reinterpret_cast<uint2*>(dst) = q;
  } else if (n == 2) {
    *reinterpret_cast<uint32_t*>(dst) = v[0] | (uint32_t(v[1]) << 16);
  } else {
    for (int i = 0; i < n; ++i) dst[i] = v[i];
  }
}

// The first n (<= 8) of v at dst: one vector store when n is 1, 2, 4 or 8 (dst
// aligned to 2 n bytes), else element stores with compile-time indices (v
// stays in registers).
__device__ __forceinline__ void store_upto8(uint16_t* dst, const uint16_t (&v)[8], int n) {
  if (n == 8 || n == 4 || n == 2) {
    store_run(dst, v, n);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < n) dst[i] = v[i];
  }
}

// Zeroes elements [c0, c1) of a BF16 row whose start is 16-byte aligned; c1 is
// a multiple of 8 (the padded reduced dimension is a multiple of 64).
__device__ __forceinline__ void zero_run(uint16_t* row, int64_t c0, int64_t c1) {
  int64_t c = c0;
  for (; c < c1 && (c & 7) != 0; ++c) row[c] = 0;
  for (; c < c1; c += 8) *reinterpret_cast<uint4*>(row + c) = make_uint4(0u, 0u, 0u, 0u);
}

// ---- split parts (see gemm_tiered) ----------------------------------------
struct StoreUpto8 {
  __device__ __forceinline__ void operator()(uint16_t* dst, const uint16_t (&v)[8], int n) const {
    store_upto8(dst, v, n);
  }
};

// Component p of group gg, one value at a time (general L).
__device__ __forceinline__ void split_part_one(uint16_t* row, int64_t gg, int p, uint16_t h, uint16_t l, int lp1,
                                               int tl, int64_t Kp_pad, int64_t Kt_pad) {
  if (tl >= lp1) {
    row[Kp_pad + gg * lp1 + p] = l;
  } else if (p < tl) {
    row[Kp_pad + gg * tl + p] = h;
    row[Kp_pad + Kt_pad + gg * tl + p] = l;
  }
}

// Zero padding of every segment of one output row.
__device__ __forceinline__ void zero_split_rows(uint16_t* row, int64_t NG, int lp1, int nsplit, int tl,
                                                int64_t Kp_pad, int64_t Kt_pad) {
  if (nsplit > 1 && tl < lp1) {
    zero_run(row, NG * lp1, Kp_pad);
    zero_run(row + Kp_pad, NG * tl, Kt_pad);
    zero_run(row + Kp_pad + Kt_pad, NG * tl, Kt_pad);
  } else {
    for (int sg = 0; sg < nsplit; ++sg) zero_run(row + sg * Kp_pad, NG * lp1, Kp_pad);
  }
}

// ---- L = 8: components in pairs ------------------------------------------
// The l+1 components of one group of eight inputs: acc[k] holds components 2k
// and 2k+1, each one FMA chain over the inputs in order (paired FMAs), with the
// kept basis values at c[t * 8 + q] (element t, component q; zero past l+1;
// 16-byte aligned shared memory, read as 16-byte broadcasts).
template <int LP1>
__device__ __forceinline__ void group8_pairs(const float (&x)[8], const float* c, float2 (&acc)[(LP1 + 1) / 2]) {
  constexpr int NP = (LP1 + 1) / 2;
#pragma unroll
  for (int k = 0; k < NP; ++k) acc[k] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const float2 xx = make_float2(x[t], x[t]);
    const float4 c0 = *reinterpret_cast<const float4*>(c + t * 8);
    acc[0] = __ffma2_rn(xx, make_float2(c0.x, c0.y), acc[0]);
    if constexpr (NP > 1) acc[NP > 1 ? 1 : 0] = __ffma2_rn(xx, make_float2(c0.z, c0.w), acc[NP > 1 ? 1 : 0]);
    if constexpr (NP > 2) {
      const float4 c1 = *reinterpret_cast<const float4*>(c + t * 8 + 4);
      acc[NP > 2 ? 2 : 0] = __ffma2_rn(xx, make_float2(c1.x, c1.y), acc[NP > 2 ? 2 : 0]);
      if constexpr (NP > 3) acc[NP > 3 ? 3 : 0] = __ffma2_rn(xx, make_float2(c1.z, c1.w), acc[NP > 3 ? 3 : 0]);
    }
  }
}

// hi = bf16(component) and lo = bf16(component - hi), two components per conversion.
template <int LP1>
__device__ __forceinline__ void split_bf16(const float2 (&acc)[(LP1 + 1) / 2], uint16_t (&hi)[8], uint16_t (&lo)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    hi[q] = 0;
    lo[q] = 0;
  }
#pragma unroll
  for (int k = 0; k < (LP1 + 1) / 2; ++k) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(acc[k].x, acc[k].y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(acc[k].x - hf.x, acc[k].y - hf.y);
    hi[2 * k] = __bfloat16_as_ushort(h.x);
    lo[2 * k] = __bfloat16_as_ushort(l.x);
    if (2 * k + 1 < LP1) {
      hi[2 * k + 1] = __bfloat16_as_ushort(h.y);
      lo[2 * k + 1] = __bfloat16_as_ushort(l.y);
    }
  }
}

// Stages the kept basis values of an L = 8 job as c[t * 8 + q] (zero past l+1)
// from the layout `at(t, q)` gives; every thread of the block calls it.
template <typename At>
__device__ __forceinline__ void stage_coef8(float* c, int lp1, At at) {
  for (int k = threadIdx.x; k < 64; k += blockDim.x) {
    const int t = k >> 3, q = k & 7;
    c[k] = q < lp1 ? at(t, q) : 0.0f;
  }
}

// ---- rows of A -> A_c (BF16, hi [+ lo]) -----------------------------------
// L = 8: one warp per two (row, run of 32 groups) units, both runs loaded before
// any arithmetic.  For each run the warp reads its 256
// inputs with lane-strided loads (each instruction reads 128 or 64 contiguous
// bytes, whatever the row's alignment), transposes them through a padded
// per-warp shared buffer (element e at e + e / 32: conflict-free both ways), and
// lane g projects group g of the run, writing its l+1 contiguous components.
// Other L (<= 64): one thread per (row, group), inputs staged in local memory.
// The thread of group 0 of a row also zeroes the row's padding columns.
// Every thread of the block reaches the one __syncthreads.
constexpr int kRowRun = 32;                         // groups per run (L = 8)
constexpr int kRowUnits = 2;                        // runs per warp, loaded together
constexpr int kRowBuf = 8 * kRowRun + 8;            // padded floats per run

template <int LP1>
__device__ __forceinline__ void rows_group8(const RowsJob& J, uint16_t* row, int64_t gg, const float (&x)[8],
                                            const float* sC) {
  float2 acc[(LP1 + 1) / 2];
  group8_pairs<LP1>(x, sC, acc);
  uint16_t hi[8], lo[8];
  split_bf16<LP1>(acc, hi, lo);
  store_upto8(row + gg * LP1, hi, LP1);
  if (J.nsplit > 1) store_split_part(row, gg, hi, lo, LP1, J.tl, J.Kp_pad, J.Kt_pad, StoreUpto8{});
}

// l+1 in {3, 5, 6, 7} without a tiered split: a run's 32 groups of components are one
// span of the row (64 (l+1) bytes from a 16-byte boundary), staged in the run's
// buffer (which the warp has read) and stored in 16-byte chunks clipped to the
// segment; lanes past the last group carry zeros.  Every lane of the warp takes part.
template <int LP1>
__device__ __forceinline__ void rows_span_odd(const RowsJob& J, const float (&x)[8], const float* sC, uint16_t* st,
                                              uint16_t* o0, int64_t room, int lane) {
  float2 acc[(LP1 + 1) / 2];
  group8_pairs<LP1>(x, sC, acc);
  uint16_t hi[8], lo[8];
  split_bf16<LP1>(acc, hi, lo);
  const int nch = static_cast<int>((room < 64 * LP1 ? room : 64 * LP1) / 16);
#pragma unroll 1
  for (int part = 0; part < (J.nsplit > 1 ? 2 : 1); ++part) {
    __syncwarp();   // the run's inputs (or the previous part) are read
#pragma unroll
    for (int p = 0; p < LP1; ++p) st[lane * LP1 + p] = part ? lo[p] : hi[p];
    __syncwarp();
    for (int k = lane; k < nch; k += 32)
      reinterpret_cast<uint4*>(o0 + part * J.Kp_pad)[k] = reinterpret_cast<const uint4*>(st)[k];
  }
}

// Warp units w0 .. w0 + kRowUnits - 1 (each a run of one row): all their loads are
// issued before any arithmetic.
template <typename InT>
__device__ __forceinline__ void rows_body8(const RowsJob& J, int64_t w0, float* sC, float* sX) {
  const int lane = threadIdx.x & 31;
  const int64_t nrun = (J.NG + kRowRun - 1) / kRowRun;
  const int lp1 = J.lp1;
  float* bufs = sX + (threadIdx.x >> 5) * (kRowUnits * kRowBuf);
#pragma unroll
  for (int v = 0; v < kRowUnits; ++v) {
    const int64_t w = w0 + v;
    const bool live = w < J.M * nrun;
    const int64_t i = live ? w / nrun : 0, run = live ? w - i * nrun : 0;
    const InT* a = static_cast<const InT*>(J.A) + i * J.lda + run * (8 * kRowRun);
    const int64_t left = J.K - run * (8 * kRowRun);
    const int nk = static_cast<int>(left < 8 * kRowRun ? left : 8 * kRowRun);
    float* buf = bufs + v * kRowBuf;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int e = s * 32 + lane;
      buf[e + s] = live && e < nk ? load_as_float(a + e) : 0.0f;
    }
  }
  stage_coef8(sC, lp1, [&](int t, int q) { return J.Cs[t * lp1 + q]; });
  __syncthreads();
  const bool odd_span = (lp1 == 3 || lp1 == 5 || lp1 == 6 || lp1 == 7) && !(J.nsplit > 1 && J.tl < lp1);
#pragma unroll 1
  for (int v = 0; v < kRowUnits; ++v) {
    const int64_t w = w0 + v;
    if (w >= J.M * nrun) break;
    const int64_t i = w / nrun, run = w - i * nrun;
    const int64_t gg = run * kRowRun + lane;
    if (odd_span) {   // the same for the whole warp
      float* fbuf = bufs + v * kRowBuf;
      float x[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) x[t] = fbuf[8 * lane + t + (lane >> 2)];
      uint16_t* row = J.Ac + i * J.pitch;
      uint16_t* o0 = row + run * (kRowRun * lp1);
      const int64_t room = 2 * (J.Kp_pad - run * (kRowRun * lp1));
      uint16_t* st = reinterpret_cast<uint16_t*>(fbuf);
      switch (lp1) {
        case 3: rows_span_odd<3>(J, x, sC, st, o0, room, lane); break;
        case 5: rows_span_odd<5>(J, x, sC, st, o0, room, lane); break;
        case 6: rows_span_odd<6>(J, x, sC, st, o0, room, lane); break;
        default: rows_span_odd<7>(J, x, sC, st, o0, room, lane); break;
      }
      if (gg == 0) zero_split_rows(row, J.NG, lp1, J.nsplit, J.tl, J.Kp_pad, J.Kt_pad);
      continue;
    }
    if (gg >= J.NG) continue;
    const float* buf = bufs + v * kRowBuf;
    float x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = buf[8 * lane + t + (lane >> 2)];
    uint16_t* row = J.Ac + i * J.pitch;
    switch (lp1) {   // the same for the whole block
      case 1: rows_group8<1>(J, row, gg, x, sC); break;
      case 2: rows_group8<2>(J, row, gg, x, sC); break;
      case 3: rows_group8<3>(J, row, gg, x, sC); break;
      case 4: rows_group8<4>(J, row, gg, x, sC); break;
      case 5: rows_group8<5>(J, row, gg, x, sC); break;
      case 6: rows_group8<6>(J, row, gg, x, sC); break;
      case 7: rows_group8<7>(J, row, gg, x, sC); break;
      default: rows_group8<8>(J, row, gg, x, sC); break;
    }
    if (gg == 0) zero_split_rows(row, J.NG, lp1, J.nsplit, J.tl, J.Kp_pad, J.Kt_pad);
  }
}

template <typename InT>
__device__ __forceinline__ void rows_body_any(const RowsJob& J, int64_t e, float* sC) {
  const bool live = e < J.M * J.NG;
  const int64_t i = live ? e / J.NG : 0, gg = live ? e - i * J.NG : 0;
  const int L = J.L, lp1 = J.lp1;
  const InT* A = static_cast<const InT*>(J.A);
  const int n = static_cast<int>(J.K - gg * L < L ? J.K - gg * L : L);
  for (int k = threadIdx.x; k < L * lp1; k += blockDim.x) sC[k] = J.Cs[k];
  __syncthreads();
  if (!live) return;
  uint16_t* out = J.Ac + i * J.pitch + gg * lp1;
  const InT* a = A + i * J.lda + gg * L;
  uint16_t* row = J.Ac + i * J.pitch;
  float xs[64];
  for (int t = 0; t < L; ++t) xs[t] = t < n ? load_as_float(a + t) : 0.0f;
  for (int p = 0; p < lp1; ++p) {
    float acc = 0.0f;
    for (int t = 0; t < L; ++t) acc = fmaf(xs[t], sC[t * lp1 + p], acc);
    const uint16_t h = bf16_bits(acc);
    out[p] = h;
    if (J.nsplit > 1) split_part_one(row, gg, p, h, bf16_bits(acc - bf16_value(h)), lp1, J.tl, J.Kp_pad, J.Kt_pad);
  }
  if (gg == 0) zero_split_rows(row, J.NG, lp1, J.nsplit, J.tl, J.Kp_pad, J.Kt_pad);
}

// Thread t of block b handles unit b * 256 + t (LT = 0), or warp units
// (b * 8 + t / 32) * kRowUnits onwards (LT = 8).
template <typename InT, int LT>
__device__ __forceinline__ void rows_body(const RowsJob& J, int64_t b, float* sC, float* sX) {
  if (LT == 8)
    rows_body8<InT>(J, (b * 8 + (threadIdx.x >> 5)) * kRowUnits, sC, sX);
  else
    rows_body_any<InT>(J, b * blockDim.x + threadIdx.x, sC);
}

template <typename InT, int LT>
__global__ void __launch_bounds__(256) project_rows_kernel(const __grid_constant__ RowsJob J) {
  __shared__ __align__(16) float sC[LT ? LT * LT : 64 * 64];
  __shared__ float sX[LT == 8 ? 8 * kRowUnits * kRowBuf : 1];
  rows_body<InT, LT>(J, blockIdx.x, sC, sX);
}


template <typename InT, int LT>
__global__ void __launch_bounds__(256) project_rows_jobs_kernel(const RowsJob* __restrict__ jobs,
                                                                const int* __restrict__ job_of) {
  __shared__ __align__(16) float sC[LT ? LT * LT : 64 * 64];
  __shared__ float sX[LT == 8 ? 8 * kRowUnits * kRowBuf : 1];
  const RowsJob& J = jobs[job_of[blockIdx.x]];
  rows_body<InT, LT>(J, static_cast<int64_t>(blockIdx.x) - J.block0, sC, sX);
}

// ---- columns of B -> B_d stored transposed (N x pitch, K-major) -----------
// One thread per (column, 4 consecutive groups): the reads of one row of B are
// coalesced across the block's columns; each thread writes 4 (l+1) contiguous
// components of its column with 16-byte stores.  The threads of the first
// group quad also zero their column's padding.
constexpr int kColGroups = 4;

// L = 8, l+1 = 4 or 8, four whole groups: the warp's 32 columns stage their
// runs in `stage` (4 KB per warp) and write them row by row (run_put_group /
// runs_write).  Every lane of the warp takes part; columns past N are not
// written back.
template <int LP1>
__device__ __forceinline__ void cols_staged(const ColsJob& J, int64_t j, int64_t g0, const float (&xa)[32],
                                            const float* sD, uint8_t* stage) {
  const int lane = threadIdx.x & 31;
  const bool live = j < J.N;
  const bool tiered = J.nsplit > 1 && J.tl < LP1, two = J.nsplit > 1 && !tiered;
  uint16_t* row = J.Bd + (live ? j : 0) * J.pitch;
  uint8_t* base = stage + (threadIdx.x >> 5) * 4096;
#pragma unroll
  for (int q = 0; q < kColGroups; ++q) {
    float x8[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x8[t] = xa[q * 8 + t];
    float2 acc[(LP1 + 1) / 2];
    group8_pairs<LP1>(x8, sD, acc);
    uint16_t hi[8], lo[8];
    split_bf16<LP1>(acc, hi, lo);
    run_put_group<LP1>(base, 128, 0, lane, q, hi);
    if (two) run_put_group<LP1>(base, 128, 1, lane, q, lo);
    if (tiered && live) store_split_part(row, g0 + q, hi, lo, LP1, J.tl, J.Kp_pad, J.Kt_pad, StoreUpto8{});
  }
  __syncwarp();
  const int64_t jw = j - lane;
  const int ncols = J.N - jw < 32 ? static_cast<int>(J.N - jw) : 32;
  uint16_t* o0 = J.Bd + jw * J.pitch + g0 * LP1;
  runs_write<LP1>(base, 128, 0, lane, o0, J.pitch, ncols);
  if (two) runs_write<LP1>(base, 128, 1, lane, o0 + J.Kp_pad, J.pitch, ncols);
  if (g0 == 0 && live) zero_split_rows(row, J.NG, LP1, J.nsplit, J.tl, J.Kp_pad, J.Kt_pad);
}

// L = 8, l+1 in {3, 5, 6, 7}, four whole groups, no tiered split: the 4 (l+1)
// components of the column's groups packed into words and stored as (l+1) 8-byte
// chunks (the run starts 8 (l+1) qd bytes into the row).
template <int LP1>
__device__ __forceinline__ void cols_quad_odd(const ColsJob& J, uint16_t* row, int64_t g0,
                                              const float (&xa)[kColGroups * 8], const float* sD) {
  uint32_t wh[2 * LP1], wl[2 * LP1];
#pragma unroll
  for (int k = 0; k < 2 * LP1; ++k) wh[k] = wl[k] = 0u;
#pragma unroll
  for (int q = 0; q < kColGroups; ++q) {
    float x8[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x8[t] = xa[q * 8 + t];
    float2 acc[(LP1 + 1) / 2];
    group8_pairs<LP1>(x8, sD, acc);
    uint16_t hi[8], lo[8];
    split_bf16<LP1>(acc, hi, lo);
#pragma unroll
    for (int p = 0; p < LP1; ++p) {
      const int e = q * LP1 + p;
      wh[e >> 1] |= uint32_t(hi[p]) << (16 * (e & 1));
      wl[e >> 1] |= uint32_t(lo[p]) << (16 * (e & 1));
    }
  }
  uint16_t* o = row + g0 * LP1;
#pragma unroll
  for (int k = 0; k < LP1; ++k) reinterpret_cast<uint2*>(o)[k] = make_uint2(wh[2 * k], wh[2 * k + 1]);
  if (J.nsplit > 1)
#pragma unroll
    for (int k = 0; k < LP1; ++k) reinterpret_cast<uint2*>(o + J.Kp_pad)[k] = make_uint2(wl[2 * k], wl[2 * k + 1]);
}

// L = 8, unstaged: group gg of one column, l+1 components.
template <int LP1>
__device__ __forceinline__ void col_group8(const ColsJob& J, uint16_t* row, int64_t gg, const float (&x8)[8],
                                           const float* sD) {
  float2 acc[(LP1 + 1) / 2];
  group8_pairs<LP1>(x8, sD, acc);
  uint16_t hi[8], lo[8];
  split_bf16<LP1>(acc, hi, lo);
  store_upto8(row + gg * LP1, hi, LP1);
  if (J.nsplit > 1) store_split_part(row, gg, hi, lo, LP1, J.tl, J.Kp_pad, J.Kt_pad, StoreUpto8{});
}

template <typename InT, int LT>
__device__ __forceinline__ void cols_body(const ColsJob& J, int64_t j, int64_t qd, float* sD, uint8_t* stage) {
  constexpr int LMAX = LT ? LT : 64;
  const int L = LT ? LT : J.L;
  const int lp1 = J.lp1;
  const bool live = j < J.N;
  const InT* B = static_cast<const InT*>(J.B);
  const int64_t g0 = qd * kColGroups;
  const int ng = static_cast<int>(J.NG - g0 < kColGroups ? J.NG - g0 : kColGroups);
  // L = 8: all kColGroups * 8 inputs are loaded before the staging barrier.
  float xa[LT == 8 ? kColGroups * 8 : 1];
  if (LT == 8) {
#pragma unroll
    for (int q = 0; q < kColGroups; ++q) {
      const int64_t k0 = (g0 + q) * 8;
      const int n = live && q < ng ? static_cast<int>(J.K - k0 < 8 ? J.K - k0 : 8) : 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) xa[q * 8 + t] = t < n ? load_as_float(B + (k0 + t) * J.ldb + j) : 0.0f;
    }
  }
  if (LT == 8)
    stage_coef8(sD, lp1, [&](int t, int q) { return J.Ds[q * 8 + t]; });
  else
    for (int k = threadIdx.x; k < L * lp1; k += blockDim.x) sD[k] = J.Ds[k];
  __syncthreads();
  if constexpr (LT == 8) {
    if (ng == kColGroups && (lp1 == 8 || lp1 == 4)) {  // the same for the whole block
      if (lp1 == 8)
        cols_staged<8>(J, j, g0, xa, sD, stage);
      else
        cols_staged<4>(J, j, g0, xa, sD, stage);
      return;
    }
  }
  if (!live) return;
  uint16_t* row = J.Bd + j * J.pitch;
  if constexpr (LT == 8) {
    if (ng == kColGroups && (lp1 == 3 || lp1 == 5 || lp1 == 6 || lp1 == 7) && !(J.nsplit > 1 && J.tl < lp1)) {
      switch (lp1) {
        case 3: cols_quad_odd<3>(J, row, g0, xa, sD); break;
        case 5: cols_quad_odd<5>(J, row, g0, xa, sD); break;
        case 6: cols_quad_odd<6>(J, row, g0, xa, sD); break;
        default: cols_quad_odd<7>(J, row, g0, xa, sD); break;
      }
      if (qd == 0) zero_split_rows(row, J.NG, lp1, J.nsplit, J.tl, J.Kp_pad, J.Kt_pad);
      return;
    }
#pragma unroll
    for (int q = 0; q < kColGroups; ++q) {
      if (q >= ng) break;
      float x8[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) x8[t] = xa[(q * 8 + t) % (LT == 8 ? kColGroups * 8 : 1)];
      switch (lp1) {   // the same for the whole block
        case 1: col_group8<1>(J, row, g0 + q, x8, sD); break;
        case 2: col_group8<2>(J, row, g0 + q, x8, sD); break;
        case 3: col_group8<3>(J, row, g0 + q, x8, sD); break;
        case 4: col_group8<4>(J, row, g0 + q, x8, sD); break;
        case 5: col_group8<5>(J, row, g0 + q, x8, sD); break;
        case 6: col_group8<6>(J, row, g0 + q, x8, sD); break;
        case 7: col_group8<7>(J, row, g0 + q, x8, sD); break;
        default: col_group8<8>(J, row, g0 + q, x8, sD); break;
      }
    }
  } else {
    for (int q = 0; q < ng; ++q) {
      const int64_t k0 = (g0 + q) * L;
      const int n = static_cast<int>(J.K - k0 < L ? J.K - k0 : L);
      float x[LMAX];
#pragma unroll
      for (int t = 0; t < LMAX; ++t)
        if (t < L) x[t] = t < n ? load_as_float(B + (k0 + t) * J.ldb + j) : 0.0f;
      for (int p = 0; p < lp1; ++p) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < LMAX; ++t)
          if (t < L) acc = fmaf(sD[p * L + t], x[t], acc);
        const uint16_t h = bf16_bits(acc);
        row[(g0 + q) * lp1 + p] = h;
        if (J.nsplit > 1)
          split_part_one(row, g0 + q, p, h, bf16_bits(acc - bf16_value(h)), lp1, J.tl, J.Kp_pad, J.Kt_pad);
      }
    }
  }
  if (qd == 0) zero_split_rows(row, J.NG, lp1, J.nsplit, J.tl, J.Kp_pad, J.Kt_pad);
}

template <typename InT, int LT>
__global__ void __launch_bounds__(256, LT == 8 ? 3 : 2) project_cols_kernel(const __grid_constant__ ColsJob J) {
  __shared__ __align__(16) float sD[LT ? LT * LT : 64 * 64];
  __shared__ __align__(16) uint8_t sStage[LT == 8 ? 8 * 4096 : 16];
  const int64_t b = blockIdx.x;
  cols_body<InT, LT>(J, (b % J.nbx) * blockDim.x + threadIdx.x, b / J.nbx, sD, sStage);
}

template <typename InT, int LT>
__global__ void __launch_bounds__(256, LT == 8 ? 3 : 2) project_cols_jobs_kernel(const ColsJob* __restrict__ jobs,
                                                                const int* __restrict__ job_of) {
  __shared__ __align__(16) float sD[LT ? LT * LT : 64 * 64];
  __shared__ __align__(16) uint8_t sStage[LT == 8 ? 8 * 4096 : 16];
  const ColsJob& J = jobs[job_of[blockIdx.x]];
  const int64_t b = static_cast<int64_t>(blockIdx.x) - J.block0;
  cols_body<InT, LT>(J, (b % J.nbx) * blockDim.x + threadIdx.x, b / J.nbx, sD, sStage);
}

// ---- FP64 path ------------------------------------------------------------
__global__ void project_rows_f64_kernel(const double* __restrict__ A, int64_t lda, int64_t M, int64_t K, int L,
                                        int lp1, int64_t NG, int64_t Kp, const double* __restrict__ Cs,
                                        double* __restrict__ Ac) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M * NG) return;
  const int64_t i = e / NG, gg = e - i * NG;
  const double* a = A + i * lda + gg * L;
  const int n = static_cast<int>(K - gg * L < L ? K - gg * L : L);
  for (int p = 0; p < lp1; ++p) {
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(a[t], Cs[t * lp1 + p], acc);
    Ac[i * Kp + gg * lp1 + p] = acc;
  }
}

__global__ void project_cols_f64_kernel(const double* __restrict__ B, int64_t ldb, int64_t N, int64_t K, int L,
                                        int lp1, int64_t NG, const double* __restrict__ Ds,
                                        double* __restrict__ Bd) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= N) return;
  for (int64_t gg = blockIdx.y; gg < NG; gg += gridDim.y) {
    const int n = static_cast<int>(K - gg * L < L ? K - gg * L : L);
    for (int p = 0; p < lp1; ++p) {
      double acc = 0.0;
      for (int t = 0; t < n; ++t) acc = fma(Ds[p * L + t], B[(gg * L + t) * ldb + j], acc);
      Bd[(gg * lp1 + p) * N + j] = acc;
    }
  }
}

// ---- CONV: signal and templates -------------------------------------------
// Box-basis form of the Haar projection with l+1 a power of two: the kept
// span is the functions constant on aligned runs of Lb = T / R samples, with
// orthonormal basis 1/sqrt(Lb) on each run.  The projected signal at
// position x is b[x] = sum_{u < Lb} s[x + u] / sqrt(Lb).  It is stored phase-
// split, with eight element shifts so every row view starts 16-byte aligned:
//   G[(sigma * Lb + phi) * P + y] = b[phi + Lb * (y + sigma)]  (0 where b is undefined).
// The templates are stored as lag-paired chunks of 64 projected components:
//   TP[c][e * 64 + t][i] = kb_t[(c - e) * 64 + i] for 0 <= c - e < R / 64, else 0,
// with kb_t[g] = sum_{u < Lb} k_t[g * Lb + u] / sqrt(Lb).
//
// One launch does both.  Signal blocks come first: block j owns the output
// columns y in [Y0, Y0 + YB) of every (sigma, phi) row, Y0 = j * YB, with
// YB = 2048 / Lb (one instantiation per Lb).  It loads s over [Lb Y0, Lb (Y0 + YB + 8)), forms the box
// sums by log2(Lb) pairwise doubling passes in shared memory (sums of 2, 4,
// ... Lb samples), and each thread writes 8 consecutive y of one (sigma, phi)
// row with one 16-byte store.  Template blocks follow (conv_template_part).
// Block 0 also clears the
// call's error word (no kernel of the call has run before it).
constexpr int kConvXB = 2048;            // box-sum positions per signal block (YB = kConvXB / Lb)
constexpr int kConvSpanMax = 64 * 40;    // samples a signal block loads: Lb (YB + 8), largest at Lb = 64
// Shared-memory index of box-sum position u: Lb floats of padding after every
// 8 Lb positions, so the reads of the output phase (lanes over phi and over
// octets 8 Lb positions apart) fall in distinct banks for every Lb.
template <int LB>
__device__ __forceinline__ int conv_pad(int u) { return u + (u / (8 * LB)) * LB; }
constexpr int kConvBuf = kConvSpanMax + kConvSpanMax / 8 + 64;  // + the over-read of the last vector

struct ConvProjParams {
  const float* s;
  int64_t S, P;
  int Lb;
  float scale;
  uint16_t* G;
  int64_t sig_blocks;
  const float* k;     // NULL: no templates in this launch
  int64_t T, nt, R;
  int Kc;
  uint16_t* TP;
  int* err;
};

template <int LB>
__device__ __forceinline__ void conv_signal_block(const ConvProjParams& p, int64_t blk, float (*buf)[kConvBuf]) {
  constexpr int YB = kConvXB / LB;
  constexpr int span = LB * (YB + 8);  // a multiple of 8; x0 too, so the span is read with 16-byte loads
  const int64_t Y0 = blk * YB;
  const int64_t x0 = Y0 * LB;
  for (int u4 = threadIdx.x; u4 < span / 4; u4 += blockDim.x) {
    const int64_t x = x0 + 4 * u4;
    float4 v;
    if (x + 4 <= p.S) {
      v = __ldg(reinterpret_cast<const float4*>(p.s + x));
    } else {
      v.x = x < p.S ? __ldg(p.s + x) : 0.0f;
      v.y = x + 1 < p.S ? __ldg(p.s + x + 1) : 0.0f;
      v.z = x + 2 < p.S ? __ldg(p.s + x + 2) : 0.0f;
      v.w = x + 3 < p.S ? __ldg(p.s + x + 3) : 0.0f;
    }
    const int u = 4 * u4;   // the four stay inside one padded run of 8 LB
    float* d = buf[0] + conv_pad<LB>(u);
    if (LB % 4 == 0) {      // the padding keeps 16-byte alignment
      *reinterpret_cast<float4*>(d) = v;
    } else {
      d[0] = v.x;
      d[1] = v.y;
      d[2] = v.z;
      d[3] = v.w;
    }
  }
  __syncthreads();
  int cur = 0;
#pragma unroll
  for (int w = 1; w < LB; w *= 2) {
    const int n = span - 2 * w + 1;  // valid sums of 2w after this pass
    if (LB >= 4) {
      // Four consecutive positions per thread (the padding keeps every
      // 4-aligned run of four contiguous and 16-byte aligned).  The last
      // vector may form up to three sums past n; they are never read.
      for (int u = 4 * threadIdx.x; u < n; u += 4 * blockDim.x) {
        const float4 a = *reinterpret_cast<const float4*>(&buf[cur][conv_pad<LB>(u)]);
        float4 r;
        if (w >= 4) {
          const float4 b = *reinterpret_cast<const float4*>(&buf[cur][conv_pad<LB>(u + w)]);
          r = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
        } else {
          const float4 b = *reinterpret_cast<const float4*>(&buf[cur][conv_pad<LB>(u + 4)]);
          const float e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
          r = make_float4(e[0] + e[w], e[1] + e[1 + w], e[2] + e[2 + w], e[3] + e[3 + w]);
        }
        *reinterpret_cast<float4*>(&buf[cur ^ 1][conv_pad<LB>(u)]) = r;
      }
    } else {
      for (int u = threadIdx.x; u < n; u += blockDim.x)
        buf[cur ^ 1][conv_pad<LB>(u)] = buf[cur][conv_pad<LB>(u)] + buf[cur][conv_pad<LB>(u + w)];
    }
    __syncthreads();
    cur ^= 1;
  }
  // BF16 once per box sum, staged transposed as bt[phi][Y - Y0] (row length
  // RL = YB + 8: 16-byte aligned rows whose stride in 16-byte units is odd).
  constexpr int RL = YB + 8;
  uint16_t* bt = reinterpret_cast<uint16_t*>(buf[cur ^ 1]);
  for (int u = threadIdx.x; u < LB * RL; u += blockDim.x) {
    const int phi = u % LB, yr = u / LB;
    const bool ok = yr < YB + 7 && x0 + u + LB <= p.S;
    bt[phi * RL + yr] = ok ? bf16_bits(buf[cur][conv_pad<LB>(u)] * p.scale) : 0;
  }
  __syncthreads();
  // Thread (octet j8, phi) holds bt[phi][8 j8 .. 8 j8 + 16) and writes the
  // eight shifted copies: copy sigma is the 8 values starting at sigma.
  static_assert(8 * LB * (YB / 8) == 8 * 256, "one (octet, phi) per thread");
  const int phi = threadIdx.x % LB, j8 = threadIdx.x / LB;
  const int64_t y0 = Y0 + 8 * j8;
  if (y0 >= p.P) return;
  const uint4* row = reinterpret_cast<const uint4*>(bt + phi * RL + 8 * j8);
  const uint4 lo4 = row[0], hi4 = row[1];
  const uint32_t w[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
  uint16_t* g = p.G + static_cast<int64_t>(phi) * p.P + y0;
  const int64_t copy_stride = static_cast<int64_t>(LB) * p.P;
#pragma unroll
  for (int sigma = 0; sigma < 8; ++sigma) {
    uint4 o;
    if (sigma % 2 == 0) {
      o = make_uint4(w[sigma / 2], w[sigma / 2 + 1], w[sigma / 2 + 2], w[sigma / 2 + 3]);
    } else {
      const int q = sigma / 2;
      o = make_uint4(__funnelshift_r(w[q], w[q + 1], 16), __funnelshift_r(w[q + 1], w[q + 2], 16),
                     __funnelshift_r(w[q + 2], w[q + 3], 16), __funnelshift_r(w[q + 3], w[q + 4], 16));
    }
    *reinterpret_cast<uint4*>(g + sigma * copy_stride) = o;
  }
}

// Template pairs.  Lb < 8: four consecutive entries of one row per thread,
// their 4 Lb samples read with Lb 16-byte loads.  Lb >= 8: one entry per
// thread, its Lb samples read with Lb / 4 independent 16-byte loads (all in
// flight at once).  The samples of a group are contiguous and 16-byte aligned.
template <int LB>
constexpr int conv_tpl_per_thread() { return LB < 8 ? 4 : 1; }

template <int LB>
__device__ __forceinline__ void conv_template_part(const ConvProjParams& p, int64_t e) {
  constexpr int EPT = conv_tpl_per_thread<LB>();
  const int64_t total = static_cast<int64_t>(p.Kc + 1) * 128 * (64 / EPT);
  if (e >= total) return;
  const int i0 = static_cast<int>(e % (64 / EPT)) * EPT;
  const int row = static_cast<int>((e / (64 / EPT)) % 128);
  const int c = static_cast<int>(e / ((64 / EPT) * 128));
  const int ee = row / 64, t = row % 64;
  const int cc = c - ee;
  float acc[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) acc[j] = 0.0f;
  // (components at or past R pad the last chunk with zeros; R is a multiple of EPT)
  if (t < p.nt && cc >= 0 && cc < p.Kc && cc * 64 + i0 < p.R) {
    const float4* kt = reinterpret_cast<const float4*>(p.k + t * p.T + (static_cast<int64_t>(cc) * 64 + i0) * LB);
    if (LB == 1) {
      const float4 v = __ldg(kt);
      acc[0] = v.x; acc[EPT > 1 ? 1 : 0] = v.y; acc[EPT > 2 ? 2 : 0] = v.z; acc[EPT > 3 ? 3 : 0] = v.w;
    } else if (LB == 2) {
      const float4 a = __ldg(kt), b = __ldg(kt + 1);
      acc[0] = a.x + a.y; acc[EPT > 1 ? 1 : 0] = a.z + a.w;
      acc[EPT > 2 ? 2 : 0] = b.x + b.y; acc[EPT > 3 ? 3 : 0] = b.z + b.w;
    } else {
      constexpr int Q = LB >= 4 ? LB / 4 : 1;  // 16-byte loads per entry
      float4 v[EPT * Q];
#pragma unroll
      for (int q = 0; q < EPT * Q; ++q) v[q] = __ldg(kt + q);
#pragma unroll
      for (int j = 0; j < EPT; ++j)
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          acc[j] += v[j * Q + q].x;
          acc[j] += v[j * Q + q].y;
          acc[j] += v[j * Q + q].z;
          acc[j] += v[j * Q + q].w;
        }
    }
  }
  uint16_t* dst = p.TP + e * EPT;
  if (EPT == 4) {
    uint16_t h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = bf16_bits(acc[j < EPT ? j : 0] * p.scale);
    store_run(dst, h, 4);
  } else {
    *dst = bf16_bits(acc[0] * p.scale);
  }
}

template <int LB>
__global__ void __launch_bounds__(256) conv_project_kernel(const __grid_constant__ ConvProjParams p) {
  __shared__ __align__(16) float buf[2][kConvBuf];
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.err = 0;
  if (blockIdx.x < p.sig_blocks)
    conv_signal_block<LB>(p, blockIdx.x, buf);
  else
    conv_template_part<LB>(p, (static_cast<int64_t>(blockIdx.x) - p.sig_blocks) * blockDim.x + threadIdx.x);
}

// ---- CONV projection for any basis (the general path) ----------------------
// Signal: G[(sigma PH + phi) P + y lp1 + p] = bf16( sum_{i<L} s[x + i] c[i, p] ) with
// x = phi + L (y + sigma): for every phase phi < L of the lags, the projections of
// the groups starting at phi + L y, all lp1 of them side by side, in copies shifted
// by sigma positions (zero extension past the signal).  Templates: the template-pair
// chunks of the box path with kd_t[g lp1 + p] = sum_{i<L} d[p, i] k_t[g L + i].
struct ConvGenParams {
  const float* s;
  int64_t S, P;
  int L, PH;
  uint16_t* G;
  int64_t sig_threads;
  const float* k;     // NULL: no templates in this launch
  int64_t T, nt, R;
  int Kc;
  uint16_t* TP;
  const float* Cs;    // L x lp1, Cs[i * lp1 + p] = c[i, p]
  const float* Ds;    // lp1 x L, Ds[p * L + i] = d[p, i]
};

template <int LP1>
__global__ void __launch_bounds__(256) conv_project_general_kernel(const __grid_constant__ ConvGenParams p) {
  __shared__ float sC[kMaxL * LP1];
  __shared__ float sD[LP1 * kMaxL];
  for (int e = threadIdx.x; e < p.L * LP1; e += blockDim.x) {
    sC[e] = p.Cs[e];
    sD[e] = p.Ds[e];
  }
  __syncthreads();
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < p.sig_threads) {
    const int64_t npos = p.P / LP1;
    const int64_t y = e % npos, rest = e / npos;
    const int phi = static_cast<int>(rest % p.PH), sigma = static_cast<int>(rest / p.PH);
    const int64_t x = phi + static_cast<int64_t>(p.L) * (y + sigma);
    float acc[LP1];
#pragma unroll
    for (int q = 0; q < LP1; ++q) acc[q] = 0.0f;
    for (int i = 0; i < p.L; ++i) {
      const float v = x + i < p.S ? __ldg(p.s + x + i) : 0.0f;
#pragma unroll
      for (int q = 0; q < LP1; ++q) acc[q] = fmaf(v, sC[i * LP1 + q], acc[q]);
    }
    uint16_t* o = p.G + (static_cast<int64_t>(sigma) * p.PH + phi) * p.P + y * LP1;
    if (LP1 >= 8) {
#pragma unroll
      for (int q = 0; q < LP1; q += 8) {
        uint16_t v8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v8[u] = bf16_bits(acc[q + u]);
        *reinterpret_cast<uint4*>(o + q) = make_uint4(v8[0] | (uint32_t(v8[1]) << 16), v8[2] | (uint32_t(v8[3]) << 16),
                                                      v8[4] | (uint32_t(v8[5]) << 16), v8[6] | (uint32_t(v8[7]) << 16));
      }
    } else {
#pragma unroll
      for (int q = 0; q < LP1; ++q) o[q] = bf16_bits(acc[q]);
    }
    return;
  }
  if (!p.k) return;
  const int64_t te = e - p.sig_threads;
  if (te >= static_cast<int64_t>(p.Kc + 1) * 128 * 64) return;
  const int i = static_cast<int>(te % 64);
  const int row = static_cast<int>((te / 64) % 128);
  const int c = static_cast<int>(te / (64 * 128));
  const int ee = row / 64, t = row % 64, cc = c - ee;
  const int64_t kk = static_cast<int64_t>(cc) * 64 + i;   // reduced component (g, q): kk = g lp1 + q
  float acc = 0.0f;
  if (t < p.nt && cc >= 0 && kk < p.R) {
    const int64_t g = kk / LP1;
    const int q = static_cast<int>(kk - g * LP1);
    const float* kt = p.k + t * p.T + g * p.L;
    for (int u = 0; u < p.L; ++u) acc = fmaf(sD[q * p.L + u], __ldg(kt + u), acc);
  }
  p.TP[te] = bf16_bits(acc);
}

}  // namespace

static cudaError_t launch_conv_project_general(const float* s, const float* k, const ConvGeom& g, uint16_t* G,
                                               uint16_t* TP, const float* Cs, const float* Ds, cudaStream_t st) {
  ConvGenParams p{};
  p.s = s;
  p.S = g.S;
  p.P = g.P;
  p.L = g.L;
  p.PH = g.PH;
  p.G = G;
  p.sig_threads = static_cast<int64_t>(g.ncopy) * g.PH * (g.P / g.lp1);
  p.k = k;
  p.T = g.T;
  p.nt = g.nt;
  p.R = g.R;
  p.Kc = g.Kc;
  p.TP = TP;
  p.Cs = Cs;
  p.Ds = Ds;
  const int64_t threads = p.sig_threads + (k ? static_cast<int64_t>(g.Kc + 1) * 128 * 64 : 0);
  const unsigned blocks = static_cast<unsigned>(ceil_div(threads, 256));
  switch (g.lp1) {   // a power of two in [1, 64]
    case 1: conv_project_general_kernel<1><<<blocks, 256, 0, st>>>(p); break;
    case 2: conv_project_general_kernel<2><<<blocks, 256, 0, st>>>(p); break;
    case 4: conv_project_general_kernel<4><<<blocks, 256, 0, st>>>(p); break;
    case 8: conv_project_general_kernel<8><<<blocks, 256, 0, st>>>(p); break;
    case 16: conv_project_general_kernel<16><<<blocks, 256, 0, st>>>(p); break;
    case 32: conv_project_general_kernel<32><<<blocks, 256, 0, st>>>(p); break;
    case 64: conv_project_general_kernel<64><<<blocks, 256, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

static unsigned grid_y(int64_t n) { return static_cast<unsigned>(n < 65535 ? (n > 0 ? n : 1) : 65535); }

RowsJob make_rows_job(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs, uint16_t* Ac) {
  RowsJob J{};
  J.A = A;
  J.Ac = Ac;
  J.Cs = Cs;
  J.lda = lda;
  J.M = g.M;
  J.K = g.K;
  J.NG = ceil_div(g.K, g.L);
  J.pitch = gemm_pitch(g);
  J.Kp_pad = g.Kp_pad;
  J.Kt_pad = g.Kt_pad;
  J.tl = g.tl;
  J.L = g.L;
  J.lp1 = g.lp1;
  J.nsplit = g.nsplit;
  J.in_bf16 = in_dtype == PJ_BF16;
  return J;
}

ColsJob make_cols_job(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds, uint16_t* Bd) {
  ColsJob J{};
  J.B = B;
  J.Bd = Bd;
  J.Ds = Ds;
  J.ldb = ldb;
  J.N = g.N;
  J.K = g.K;
  J.NG = ceil_div(g.K, g.L);
  J.pitch = gemm_pitch(g);
  J.Kp_pad = g.Kp_pad;
  J.Kt_pad = g.Kt_pad;
  J.tl = g.tl;
  J.nbx = ceil_div(g.N, 256);
  J.L = g.L;
  J.lp1 = g.lp1;
  J.nsplit = g.nsplit;
  J.in_bf16 = in_dtype == PJ_BF16;
  return J;
}

int64_t rows_job_blocks(const RowsJob& J) {
  return J.L == 8 ? ceil_div(J.M * ceil_div(J.NG, kRowRun), 8 * kRowUnits) : ceil_div(J.M * J.NG, 256);
}
int64_t cols_job_blocks(const ColsJob& J) { return J.nbx * ceil_div(J.NG, kColGroups); }

int projection_class(int in_bf16, int L) { return (in_bf16 ? 2 : 0) + (L == 8 ? 1 : 0); }

cudaError_t launch_project_rows_simt(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs,
                                     uint16_t* Ac, cudaStream_t st) {
  if (g.M == 0 || g.K == 0) return cudaSuccess;
  const RowsJob J = make_rows_job(A, lda, in_dtype, g, Cs, Ac);
  const unsigned blocks = static_cast<unsigned>(rows_job_blocks(J));
  switch (projection_class(J.in_bf16, J.L)) {
    case 0: project_rows_kernel<float, 0><<<blocks, 256, 0, st>>>(J); break;
    case 1: project_rows_kernel<float, 8><<<blocks, 256, 0, st>>>(J); break;
    case 2: project_rows_kernel<__nv_bfloat16, 0><<<blocks, 256, 0, st>>>(J); break;
    default: project_rows_kernel<__nv_bfloat16, 8><<<blocks, 256, 0, st>>>(J); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_project_cols_simt(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds,
                                     uint16_t* Bd, cudaStream_t st) {
  if (g.N == 0 || g.K == 0) return cudaSuccess;
  const ColsJob J = make_cols_job(B, ldb, in_dtype, g, Ds, Bd);
  const unsigned blocks = static_cast<unsigned>(cols_job_blocks(J));
  switch (projection_class(J.in_bf16, J.L)) {
    case 0: project_cols_kernel<float, 0><<<blocks, 256, 0, st>>>(J); break;
    case 1: project_cols_kernel<float, 8><<<blocks, 256, 0, st>>>(J); break;
    case 2: project_cols_kernel<__nv_bfloat16, 0><<<blocks, 256, 0, st>>>(J); break;
    default: project_cols_kernel<__nv_bfloat16, 8><<<blocks, 256, 0, st>>>(J); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_project_rows_jobs(int cls, const RowsJob* jobs, const int* job_of, int64_t blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  const unsigned nb = static_cast<unsigned>(blocks);
  switch (cls) {
    case 0: project_rows_jobs_kernel<float, 0><<<nb, 256, 0, st>>>(jobs, job_of); break;
    case 1: project_rows_jobs_kernel<float, 8><<<nb, 256, 0, st>>>(jobs, job_of); break;
    case 2: project_rows_jobs_kernel<__nv_bfloat16, 0><<<nb, 256, 0, st>>>(jobs, job_of); break;
    default: project_rows_jobs_kernel<__nv_bfloat16, 8><<<nb, 256, 0, st>>>(jobs, job_of); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_project_cols_jobs(int cls, const ColsJob* jobs, const int* job_of, int64_t blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  const unsigned nb = static_cast<unsigned>(blocks);
  switch (cls) {
    case 0: project_cols_jobs_kernel<float, 0><<<nb, 256, 0, st>>>(jobs, job_of); break;
    case 1: project_cols_jobs_kernel<float, 8><<<nb, 256, 0, st>>>(jobs, job_of); break;
    case 2: project_cols_jobs_kernel<__nv_bfloat16, 0><<<nb, 256, 0, st>>>(jobs, job_of); break;
    default: project_cols_jobs_kernel<__nv_bfloat16, 8><<<nb, 256, 0, st>>>(jobs, job_of); break;
  }
  return cudaGetLastError();
}


cudaError_t launch_project_rows_f64(const double* A, int64_t lda, const GemmGeom& g, const double* Cs, double* Ac,
                                    cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (g.M == 0 || NG == 0) return cudaSuccess;
  project_rows_f64_kernel<<<static_cast<unsigned>(ceil_div(g.M * NG, 128)), 128, 0, st>>>(A, lda, g.M, g.K, g.L,
                                                                                          g.lp1, NG, g.Kp, Cs, Ac);
  return cudaGetLastError();
}

cudaError_t launch_project_cols_f64(const double* B, int64_t ldb, const GemmGeom& g, const double* Ds, double* Bd,
                                    cudaStream_t st) {
  const int64_t NG = ceil_div(g.K, g.L);
  if (g.N == 0 || NG == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(ceil_div(g.N, 128)), grid_y(NG));
  project_cols_f64_kernel<<<grid, 128, 0, st>>>(B, ldb, g.N, g.K, g.L, g.lp1, NG, Ds, Bd);
  return cudaGetLastError();
}

cudaError_t launch_conv_project(const float* s, const float* k, const ConvGeom& g, uint16_t* G, uint16_t* TP,
                                int* err, cudaStream_t st, const float* Cs, const float* Ds) {
  if (!g.box) return launch_conv_project_general(s, k, g, G, TP, Cs, Ds, st);
  ConvProjParams p{};
  p.s = s;
  p.S = g.S;
  p.P = g.P;
  p.Lb = g.Lb;
  p.scale = 1.0f / sqrtf(static_cast<float>(g.Lb));
  p.G = G;
  p.sig_blocks = ceil_div(g.P, kConvXB / g.Lb);
  p.k = k;
  p.T = g.T;
  p.nt = g.nt;
  p.R = g.R;
  p.Kc = g.Kc;
  p.TP = TP;
  p.err = err;
  const int64_t tpl_threads = static_cast<int64_t>(g.Kc + 1) * 128 * (g.Lb < 8 ? 16 : 64);
  const int64_t tpl_blocks = k ? ceil_div(tpl_threads, 256) : 0;
  const unsigned blocks = static_cast<unsigned>(p.sig_blocks + tpl_blocks);
  switch (g.Lb) {  // Lb = T / R is a power of two in [1, 64]
    case 1: conv_project_kernel<1><<<blocks, 256, 0, st>>>(p); break;
    case 2: conv_project_kernel<2><<<blocks, 256, 0, st>>>(p); break;
    case 4: conv_project_kernel<4><<<blocks, 256, 0, st>>>(p); break;
    case 8: conv_project_kernel<8><<<blocks, 256, 0, st>>>(p); break;
    case 16: conv_project_kernel<16><<<blocks, 256, 0, st>>>(p); break;
    case 32: conv_project_kernel<32><<<blocks, 256, 0, st>>>(p); break;
    case 64: conv_project_kernel<64><<<blocks, 256, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pj
