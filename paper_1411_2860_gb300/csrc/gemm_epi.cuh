// Epilogue helpers shared by the reduced-GEMM kernels (gemm_tc.cu, gemm_cg2.cu):
// the expansion of a gradient product's components back to samples, written
// straight from the registers that tcgen05.ld filled (ExpandArgs, common.hpp).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "common.hpp"
#include "tc.cuh"

namespace pj {
namespace {

template <bool kBF16>
__device__ __forceinline__ void store_run(void* out, int64_t off, const float (&y)[8], int n, int per) {
  if (kBF16) {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + off;
    if (n == per && per >= 2) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        w[k] = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(y[2 * k]))) |
               (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(y[2 * k + 1]))) << 16);
      if (per == 8) *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
      else if (per == 4) *reinterpret_cast<uint2*>(o) = make_uint2(w[0], w[1]);
      else *reinterpret_cast<uint32_t*>(o) = w[0];
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < n) o[t] = __float2bfloat16_rn(y[t]);
    }
  } else {
    float* o = static_cast<float*>(out) + off;
    if (n == per && per >= 4) {
      reinterpret_cast<float4*>(o)[0] = make_float4(y[0], y[1], y[2], y[3]);
      if (per == 8) reinterpret_cast<float4*>(o)[1] = make_float4(y[4], y[5], y[6], y[7]);
    } else if (n == per && per == 2) {
      *reinterpret_cast<float2*>(o) = make_float2(y[0], y[1]);
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < n) o[t] = y[t];
    }
  }
}

// The expansion runs over 8 TMEM columns at a time in a loop that is not
// unrolled: a fully unrolled 32-column step is several KB of straight-line
// code per (mode, l+1, dtype), and with one epilogue warp per scheduler the
// instruction fetch, not the stores, then bounds the epilogue.

// Mode 1 (components on the TMEM lanes): lane `lane` holds component p = kk % LP1
// of group g = kk / LP1 for 8 output rows i0 .. i0 + 7; the LP1 lanes of a group
// exchange their values and each writes 8 / LP1 of the group's 8 samples per row.
template <int LP1, bool kBF16>
__device__ __forceinline__ void expand_rows_x8(const uint32_t (&r)[8], int lane, int kk, int Kp, int i0, int M,
                                               const ExpandArgs& ex, const float* sc) {
  constexpr int per = 8 / LP1;
  const int g = kk / LP1, pc = kk - g * LP1, t0 = pc * per;
  const int lbase = lane & ~(LP1 - 1);
  const int64_t col0 = static_cast<int64_t>(g) * 8 + t0;
  void* const out = ex.out;
  const int64_t ld = ex.ld;
  int n = static_cast<int>(ex.K - col0);
  n = kk < Kp ? (n < 0 ? 0 : (n > per ? per : n)) : 0;
  float cf[per][LP1];
#pragma unroll
  for (int t = 0; t < per; ++t)
#pragma unroll
    for (int pp = 0; pp < LP1; ++pp) cf[t][pp] = sc[(t0 + t) * LP1 + pp];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    float v[LP1];
#pragma unroll
    for (int pp = 0; pp < LP1; ++pp) v[pp] = __shfl_sync(0xffffffffu, __uint_as_float(r[u]), lbase + pp);
    if (n > 0 && i0 + u < M) {
      float y[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float acc = 0.0f;
        if (t < per) {
#pragma unroll
          for (int pp = 0; pp < LP1; ++pp) acc = fmaf(v[pp], cf[t < per ? t : 0][pp], acc);
        }
        y[t] = acc;
      }
      store_run<kBF16>(out, static_cast<int64_t>(i0 + u) * ld + col0, y, n, per);
    }
  }
}

// Mode 2 (components on the TMEM columns): this thread holds components
// k0 .. k0 + 7 of output column j; each group of LP1 gives 8 sample rows.
// The 8 x LP1 coefficients sit in registers for LP1 <= 4 (read from shared
// memory per use for LP1 = 8, where they would take 64 registers).
template <int LP1, bool kBF16>
__device__ __forceinline__ void expand_cols_x8(const uint32_t (&r)[8], int k0, int Kp, int j,
                                               const ExpandArgs& ex, const float* sd) {
  constexpr bool kRegs = LP1 <= 4;
  float cr[kRegs ? LP1 * 8 : 1];
  if (kRegs) {
#pragma unroll
    for (int e = 0; e < (kRegs ? LP1 * 8 : 1); ++e) cr[e] = sd[e];
  }
  const int64_t ld = ex.ld, K = ex.K;
  auto* out = static_cast<typename std::conditional<kBF16, __nv_bfloat16, float>::type*>(ex.out);
#pragma unroll
  for (int a = 0; a < 8 / LP1; ++a) {
    const int kk = k0 + a * LP1;
    if (kk >= Kp) break;
    const int64_t row0 = static_cast<int64_t>(kk / LP1) * 8;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (row0 + t >= K) break;
      float acc = 0.0f;
#pragma unroll
      for (int pp = 0; pp < LP1; ++pp)
        acc = fmaf(kRegs ? cr[kRegs ? pp * 8 + t : 0] : sd[pp * 8 + t], __uint_as_float(r[a * LP1 + pp]), acc);
      const int64_t off = (row0 + t) * ld + j;
      if (kBF16)
        out[off] = __float2bfloat16_rn(acc);
      else
        out[off] = acc;
    }
  }
}

template <int LP1, bool kBF16>
__device__ __noinline__ void expand_tile_cols(uint32_t taddr, int ncols, const ExpandArgs ex, const float* sc,
                                              int lane, int kk_lane, int Kp, int i0, int M, int j, bool jok) {
#pragma unroll 1
  for (int c = 0; c < ncols; c += 8) {
    uint32_t r[8];
    tmem_ld_x8(taddr + c, r);
    tmem_wait_ld();
    if (ex.mode == 1) {
      if (i0 + c < M) expand_rows_x8<LP1, kBF16>(r, lane, kk_lane, Kp, i0 + c, M, ex, sc);
    } else if (jok && i0 + c < Kp) {
      expand_cols_x8<LP1, kBF16>(r, i0 + c, Kp, j, ex, sc);
    }
  }
}

// Expands `ncols` (a multiple of 8) TMEM columns starting at taddr (this warp's
// lane quadrant), whose first column is output row i0 (mode 1: the lanes hold
// components kk_lane of Kp) or component i0 of Kp (mode 2: the lanes hold output
// column j).
__device__ __forceinline__ void expand_tile(uint32_t taddr, int ncols, const ExpandArgs& ex, const float* s_coef,
                                            int lane, int kk_lane, int Kp, int i0, int M, int j, bool jok) {
  if (ex.out_bf16) {
    switch (ex.lp1) {
      case 1: expand_tile_cols<1, true>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
      case 2: expand_tile_cols<2, true>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
      case 4: expand_tile_cols<4, true>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
      default: expand_tile_cols<8, true>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
    }
  } else {
    switch (ex.lp1) {
      case 1: expand_tile_cols<1, false>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
      case 2: expand_tile_cols<2, false>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
      case 4: expand_tile_cols<4, false>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
      default: expand_tile_cols<8, false>(taddr, ncols, ex, s_coef, lane, kk_lane, Kp, i0, M, j, jok); break;
    }
  }
}

}  // namespace
}  // namespace pj
