// E4M3 with per-32 UE8M0 block scales (the "FP8 E4M3 with per-block scales" of
// the reduced products): the scale exponent of a run, the E4M3 rounding of a
// pair of values, and where a run's scale byte sits in the block-scale layout
// gemm_mx_kernel reads.  Shared by the quantiser pass (gemm_mx.cu) and the
// projection kernel that writes E4M3 components itself (project_tma.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.hpp"

namespace pj {

// e = ceil(log2(amax / 448)) from the bits of amax, clamped to the UE8M0 range
// (448 is the largest E4M3 value, so amax / 2^e never saturates).
__device__ __forceinline__ int mx_exponent(float amax) {
  if (!(amax > 0.0f)) return 0;
  const uint32_t b = __float_as_uint(amax);
  const int E = static_cast<int>((b >> 23) & 255u) - 127;
  const int e = E - 8 + ((b & 0x7FFFFFu) > 0x600000u ? 1 : 0);
  return e < -127 ? -127 : (e > 127 ? 127 : e);
}

// E4M3 (round to nearest even, finite) of (a, b) * inv: byte of a low, of b high.
__device__ __forceinline__ uint32_t e4m3x2(float a, float b, float inv) {
  return static_cast<uint32_t>(__nv_cvt_float2_to_fp8x2(make_float2(a * inv, b * inv), __NV_SATFINITE, __NV_E4M3));
}

// The two values of an E4M3 pair (as e4m3x2 packs them).
__device__ __forceinline__ float2 e4m3x2_value(uint32_t q) {
  return __half22float2(
      __half2(__nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(q & 0xFFFFu), __NV_E4M3)));
}

// Byte of the scale of run cg (32 components) of row r: per tile of rows and
// 128-component stage, row r of a 128-row group and K block b at byte
// (r % 32) * 16 + (r / 32) * 4 + b.
__device__ __forceinline__ int64_t mx_sf_offset(const MxQuantSide& a, int64_t r, int64_t cg) {
  const int64_t tile = r / a.tile_rows, rr = r - tile * a.tile_rows;
  const int64_t atom = rr >> 7, ar = rr & 127;
  return ((tile * a.sf_stages + (cg >> 2)) * a.atoms + atom) * 512 + (ar & 31) * 16 + (ar >> 5) * 4 + (cg & 3);
}

}  // namespace pj
