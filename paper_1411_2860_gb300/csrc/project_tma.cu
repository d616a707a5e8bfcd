// TMA-staged projection of GEMM operands for groups of L = 8 (Sec. III-B,
// Fig. 5): the rows of A are multiplied group-wise by the kept columns of C,
// the columns of B by the kept rows of D = C^-1, and the (l+1) components of
// every group are written as BF16 (hi, and for the split precision also
// lo = the rounding residual) in the group-major order of the reduced inner
// dimension, or as E4M3 with per-32 block scales (mx.cuh).
//
// The work is HBM-bound streaming.  One persistent launch (as many blocks per
// SM as fit: two for FP32 inputs, three for BF16) projects both operands: its
// units are the 32 x 256-element tiles of A followed by those of B.  Each
// block keeps a ring of tiles in flight (three stages of 32 KB for FP32
// inputs, four of 16 KB for BF16) with 2D TMA loads
// (zero fill past the edges supplies the zero extension of a short last
// group), issued by its thread 0, and its eight
// warps project each tile out of shared memory.  The batched form (many
// operands per launch) also reads operands whose row pitch TMA cannot address,
// one bulk copy per tile row.  Every wait is bounded; on a timeout the kernel
// records an error code, lets the copies it issued land and returns.
#include <cuda_bf16.h>

#include <cstring>

#include "common.hpp"
#include "mx.cuh"
#include "tc.cuh"
#include "tmap.hpp"

namespace pj {
namespace {

constexpr int kPtConsumers = 256;
constexpr int kPtThreads = kPtConsumers;     // thread 0 also issues the copies
constexpr int kPtStages = 3;
constexpr int kPtBoxX = 256;  // elements along the contiguous dimension
constexpr int kPtBoxY = 32;   // rows
constexpr int kPtTileMax = kPtBoxX * kPtBoxY * 4;

// One operand of the launch: side 0 = rows of A, side 1 = columns of B.
struct ProjSide {
  const float* coef;    // rows: C kept columns at [t * lp1 + p]; cols: D kept rows at [p * 8 + t]
  uint16_t* out;        // rows: A_c (M x pitch); cols: B_d (N x pitch)
  int64_t n_out;        // rows: M; cols: N
  int64_t num_units;    // 0 when this operand is not part of the launch
  int units_x, units_y;
  int tile_bytes;
};

struct ProjTmaParams {
  CUtensorMap map[2];   // A: dims {K, M}; B: dims {N, K}; box {256, 32}
  ProjSide side[2];
  MxQuantSide q[2];     // E4M3 instantiations: where each side's components and block scales go
  int64_t pitch, Kp_pad, Kt_pad;
  int64_t NG;           // groups along K
  int nsplit, tl;
  int* err;
};

// What a consumer needs to place the components of one tile.
struct TileCtx {
  uint16_t* out;
  int64_t n_out, NG, pitch, Kp_pad, Kt_pad;
  int units_x, units_y, nsplit, tl;
};

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return a | (uint32_t(b) << 16); }

// Writes the first n of v[0..7] at dst (dst aligned to 2 n bytes when n is 1, 2, 4 or 8).
__device__ __forceinline__ void store_upto8(uint16_t* dst, const uint16_t (&v)[8], int n) {
  if (n == 8) {
    *reinterpret_cast<uint4*>(dst) = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]),
                                                pack2(v[6], v[7]));
  } else if (n == 4) {
    *reinterpret_cast<uint2*>(dst) = make_uint2(pack2(v[0], v[1]), pack2(v[2], v[3]));
  } else if (n == 2) {
    *reinterpret_cast<uint32_t*>(dst) = pack2(v[0], v[1]);
  } else {
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (p < n) dst[p] = v[p];
  }
}

__device__ __forceinline__ void zero_tail(uint16_t* row, int64_t c0, int64_t c1) {
  int64_t c = c0;
  for (; c < c1 && (c & 7) != 0; ++c) row[c] = 0;
  for (; c < c1; c += 8) *reinterpret_cast<uint4*>(row + c) = make_uint4(0u, 0u, 0u, 0u);
}

// Padding of every segment of one output row (see gemm_tiered for the layout).
__device__ __forceinline__ void zero_row_tails(const TileCtx& c, uint16_t* row, int lp1) {
  if (c.nsplit > 1 && c.tl < lp1) {
    zero_tail(row, c.NG * lp1, c.Kp_pad);
    zero_tail(row + c.Kp_pad, c.NG * c.tl, c.Kt_pad);
    zero_tail(row + c.Kp_pad + c.Kt_pad, c.NG * c.tl, c.Kt_pad);
  } else {
    for (int sg = 0; sg < c.nsplit; ++sg) zero_tail(row + sg * c.Kp_pad, c.NG * lp1, c.Kp_pad);
  }
}

// Eight consecutive inputs of one group from a shared-memory tile row, as four
// pairs (x[2t], x[2t+1]) for the paired FMAs below.
template <typename InT>
__device__ __forceinline__ void tile_group8(const uint8_t* row, int g, float2 (&x)[4]);

template <>
__device__ __forceinline__ void tile_group8<float>(const uint8_t* row, int g, float2 (&x)[4]) {
  // Lanes 4..7 of every quarter warp read their second 16 bytes first, so the
  // eight 16-byte reads of a quarter warp cover all 32 banks once.
  const float4* p = reinterpret_cast<const float4*>(row + g * 32);
  const int h = (g >> 2) & 1;
  const float4 a = p[h], b = p[h ^ 1];
  const float4 lo = h ? b : a, hi = h ? a : b;
  x[0] = make_float2(lo.x, lo.y);
  x[1] = make_float2(lo.z, lo.w);
  x[2] = make_float2(hi.x, hi.y);
  x[3] = make_float2(hi.z, hi.w);
}

template <>
__device__ __forceinline__ void tile_group8<__nv_bfloat16>(const uint8_t* row, int g, float2 (&x)[4]) {
  const uint4 u = *reinterpret_cast<const uint4*>(row + g * 16);
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) x[t] = make_float2(__uint_as_float(w[t] << 16), __uint_as_float(w[t] & 0xffff0000u));
}

__device__ __forceinline__ float row_elem(const uint8_t* row, int j, float*) {
  return reinterpret_cast<const float*>(row)[j];
}
__device__ __forceinline__ float row_elem(const uint8_t* row, int j, __nv_bfloat16*) {
  return __uint_as_float(uint32_t(reinterpret_cast<const uint16_t*>(row)[j]) << 16);
}

// Group g of a row that starts sb bytes past the 16-byte aligned `row` (sb a
// multiple of the element size, the same for the whole warp): the aligned
// 16-byte words that cover it are read and the eight elements picked from them
// with compile-time indices, one branch per offset.
template <int S>
__device__ __forceinline__ void pick8(const float (&v)[12], float2 (&x)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) x[t] = make_float2(v[S + 2 * t], v[S + 2 * t + 1]);
}

__device__ __forceinline__ void row_group8_at(const uint8_t* row, int g, int sb, float2 (&x)[4], float*) {
  const float4* p = reinterpret_cast<const float4*>(row) + 2 * g;
  const int h = (g >> 2) & 1;   // (the bank order of tile_group8)
  const float4 a0 = p[h], a1 = p[h ^ 1];
  const float4 a = h ? a1 : a0, b = h ? a0 : a1;
  float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (sb != 0) c = p[2];
  const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
  switch (sb >> 2) {
    case 0: pick8<0>(v, x); break;
    case 1: pick8<1>(v, x); break;
    case 2: pick8<2>(v, x); break;
    default: pick8<3>(v, x); break;
  }
}

template <int S>
__device__ __forceinline__ void pick8_bf16(const uint32_t (&w)[8], float2 (&x)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t u = (S & 1) ? __funnelshift_r(w[S / 2 + k], w[S / 2 + k + 1], 16) : w[S / 2 + k];
    x[k] = make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  }
}

__device__ __forceinline__ void row_group8_at(const uint8_t* row, int g, int sb, float2 (&x)[4], __nv_bfloat16*) {
  const uint4* p = reinterpret_cast<const uint4*>(row) + g;
  const uint4 u0 = p[0];
  uint4 u1 = make_uint4(0u, 0u, 0u, 0u);
  if (sb != 0) u1 = p[1];
  const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
  switch (sb >> 1) {
    case 0: pick8_bf16<0>(w, x); break;
    case 1: pick8_bf16<1>(w, x); break;
    case 2: pick8_bf16<2>(w, x); break;
    case 3: pick8_bf16<3>(w, x); break;
    case 4: pick8_bf16<4>(w, x); break;
    case 5: pick8_bf16<5>(w, x); break;
    case 6: pick8_bf16<6>(w, x); break;
    default: pick8_bf16<7>(w, x); break;
  }
}

// Where the consumers find a tile.  A TMA tile holds 32 dense rows of 256
// elements, zeros past the operand's edges.  A bulk tile (an operand whose row
// pitch TMA cannot address; each row copied on its own from the 16-byte granule
// that holds its first element) has rows of 256 elements + 16 bytes, row e
// starting shift(e) bytes in (its source's offset within the granule), and
// nothing past the operand's `rows` rows and `cols` columns: the consumers read
// zeros there.
template <typename InT, bool kBulk>
struct TileIn {
  static constexpr int kRowBytes = kPtBoxX * static_cast<int>(sizeof(InT)) + (kBulk ? 16 : 0);
  uint8_t* base;
  int a0, ldm;       // bulk: row 0's offset in its granule; the row pitch in bytes mod 16
  int rows, cols;    // bulk: rows and columns of the tile inside the operand
  // (ldm is a multiple of 2, so the offsets repeat every 8 rows)
  __device__ __forceinline__ int shift(int e) const { return kBulk ? (a0 + (e & 7) * ldm) & 15 : 0; }
  __device__ __forceinline__ float elem(int e, int j) const {
    if (kBulk && e >= rows) return 0.0f;
    return row_elem(base + e * kRowBytes + shift(e), j, static_cast<InT*>(nullptr));
  }
  // the eight elements of group g of row e
  __device__ __forceinline__ void group8(int e, int g, float2 (&x)[4]) const {
    if (!kBulk) {
      tile_group8<InT>(base + e * kRowBytes, g, x);
      return;
    }
    row_group8_at(base + e * kRowBytes, g, shift(e), x, static_cast<InT*>(nullptr));
    if (cols < kPtBoxX) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (8 * g + 2 * t >= cols) x[t].x = 0.0f;
        if (8 * g + 2 * t + 1 >= cols) x[t].y = 0.0f;
      }
    }
  }
};

// The kept basis vectors, coef[q * 8 + t] (component q, element t of the group),
// read as pairs (t, t+1).  With kRegs a tile loads them into registers once
// (rows: every l+1; columns: l+1 <= 4, whose threads already hold 32 inputs);
// otherwise every use reads shared memory or (kG) global memory through the L1
// cache.
template <int LP1, bool kG, bool kRegsWanted = true>
struct PtCoef {
  static constexpr bool kRegs = kRegsWanted;
  float2 c[kRegs ? LP1 : 1][4];
  const float* src;
  __device__ __forceinline__ explicit PtCoef(const float* coef) : src(coef) {
    if (kRegs) {
#pragma unroll
      for (int q = 0; q < (kRegs ? LP1 : 1); ++q)
#pragma unroll
        for (int t = 0; t < 4; ++t) c[q][t] = load(q, t);
    }
  }
  __device__ __forceinline__ float2 load(int q, int t) const {
    const float2* p = reinterpret_cast<const float2*>(src + q * 8) + t;
    return kG ? __ldg(p) : *p;
  }
  __device__ __forceinline__ float2 get(int q, int t) const { return kRegs ? c[kRegs ? q : 0][t] : load(q, t); }
};

// Component q of a group: with register-held coefficients the eight products
// summed as two interleaved chains of paired FMAs (even and odd elements), then
// added.
template <int LP1, bool kG, bool kR>
__device__ __forceinline__ float project_one(const float2 (&x)[4], const PtCoef<LP1, kG, kR>& cf, int q) {
  if (kR) {
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int t = 0; t < 4; ++t) acc = __ffma2_rn(x[t], cf.get(q, t), acc);
    return acc.x + acc.y;
  }
  // otherwise two 16-byte reads per component and one chain of scalar FMAs, which
  // keeps the 8 (l+1) coefficients out of registers
  const float4* p4 = reinterpret_cast<const float4*>(cf.src + q * 8);
  const float4 u = kG ? __ldg(p4) : p4[0];
  const float4 v = kG ? __ldg(p4 + 1) : p4[1];
  float acc = 0.0f;
  acc = fmaf(x[0].x, u.x, acc);
  acc = fmaf(x[0].y, u.y, acc);
  acc = fmaf(x[1].x, u.z, acc);
  acc = fmaf(x[1].y, u.w, acc);
  acc = fmaf(x[2].x, v.x, acc);
  acc = fmaf(x[2].y, v.y, acc);
  acc = fmaf(x[3].x, v.z, acc);
  acc = fmaf(x[3].y, v.w, acc);
  return acc;
}

template <int LP1, bool kG, bool kR>
__device__ __forceinline__ void project8(const float2 (&x)[4], const PtCoef<LP1, kG, kR>& cf, bool need_lo,
                                         uint16_t (&hi)[8], uint16_t (&lo)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    hi[q] = 0;
    lo[q] = 0;
  }
#pragma unroll
  for (int q = 0; q < LP1; ++q) {
    const float acc = project_one(x, cf, q);
    hi[q] = bf16_bits(acc);
    if (need_lo) lo[q] = bf16_bits(acc - bf16_value(hi[q]));
  }
}

// Tiered split: hi of every kept component into hi[], and for the lead
// components q < tl the hi and lo terms straight to their segments (lh, ll),
// so no array of lo terms stays live.
template <int LP1, bool kG, bool kR>
__device__ __forceinline__ void project8_lead(const float2 (&x)[4], const PtCoef<LP1, kG, kR>& cf, uint16_t (&hi)[8],
                                              int tl, bool valid, uint16_t* lh, uint16_t* ll) {
#pragma unroll
  for (int q = 0; q < 8; ++q) hi[q] = 0;
#pragma unroll
  for (int q = 0; q < LP1; ++q) {
    const float acc = project_one(x, cf, q);
    hi[q] = bf16_bits(acc);
    if (valid && q < tl) {
      lh[q] = hi[q];
      ll[q] = bf16_bits(acc - bf16_value(hi[q]));
    }
  }
}

// l+1 whose runs of components are neither one vector nor whole 16-byte chunks.
template <int LP1>
constexpr bool kOddRun = LP1 == 3 || LP1 == 5 || LP1 == 6 || LP1 == 7;

// Rows: tile = 32 rows of A x 256 elements (32 groups).  Warp w projects rows
// w, w+8, w+16, w+24; lane g the tile's group g, so a warp writes one run of
// 32 (l+1) contiguous components per row.
template <typename InT, int LP1, bool kG, bool kTiered>
__device__ __forceinline__ void rows_tile(const TileCtx& c, const TileIn<InT, false>& tin, const float* sCoef, int ux,
                                          int uy) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gg = static_cast<int64_t>(ux) * 32 + lane;
  const PtCoef<LP1, kG, !(kG && LP1 == 8)> cf(sCoef);   // (as in rows_tile_q)
  const bool need_lo = c.nsplit > 1;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = static_cast<int64_t>(uy) * kPtBoxY + warp + 8 * u;
    float2 x[4];
    tin.group8(warp + 8 * u, lane, x);
    if (kTiered) {
      const bool valid = i < c.n_out && gg < c.NG;
      uint16_t* row = c.out + (valid ? i : 0) * c.pitch;
      uint16_t hi[8];
      project8_lead(x, cf, hi, c.tl, valid, row + c.Kp_pad + gg * c.tl,
                             row + c.Kp_pad + c.Kt_pad + gg * c.tl);
      if (valid) store_upto8(row + gg * LP1, hi, LP1);
    } else {
      uint16_t hi[8], lo[8];
      project8(x, cf, need_lo, hi, lo);
      if constexpr (kOddRun<LP1>) {
        // The warp's 32 runs of l+1 components are one span of the output row, 64 (l+1)
        // bytes from a 16-byte boundary: staged in this row's slice of the tile (read by
        // this warp alone, and read already) and stored in 16-byte chunks, clipped to
        // the segment (lanes past the last group carry the zeros of the TMA fill).
        if (i < c.n_out) {   // the same for the whole warp
          uint16_t* st = reinterpret_cast<uint16_t*>(tin.base + (warp + 8 * u) * TileIn<InT, false>::kRowBytes);
          const int64_t c0 = static_cast<int64_t>(ux) * 32 * LP1;
          const int64_t room = 2 * (c.Kp_pad - c0);
          const int nch = static_cast<int>((room < 64 * LP1 ? room : 64 * LP1) / 16);
          uint16_t* o0 = c.out + i * c.pitch + c0;
#pragma unroll 1
          for (int part = 0; part < (need_lo ? 2 : 1); ++part) {
            __syncwarp();   // the row's inputs (or the previous part) are read
#pragma unroll
            for (int p = 0; p < LP1; ++p) st[lane * LP1 + p] = part ? lo[p] : hi[p];
            __syncwarp();
            for (int k = lane; k < nch; k += 32)
              reinterpret_cast<uint4*>(o0 + part * c.Kp_pad)[k] = reinterpret_cast<const uint4*>(st)[k];
          }
        }
      } else if (i < c.n_out && gg < c.NG) {
        uint16_t* o = c.out + i * c.pitch + gg * LP1;
        store_upto8(o, hi, LP1);
        if (c.nsplit > 1) store_upto8(o + c.Kp_pad, lo, LP1);
      }
    }
  }
  // staging writes before the stage's next TMA fill
  if constexpr (kOddRun<LP1> && !kTiered) fence_proxy_async_smem();
  if (ux == c.units_x - 1 && lane == 0) {
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
      const int64_t i = static_cast<int64_t>(uy) * kPtBoxY + warp + 8 * u;
      if (i < c.n_out) zero_row_tails(c, c.out + i * c.pitch, LP1);
    }
  }
}

// E4M3 components with per-32 UE8M0 block scales written by the projection
// itself (the quantiser's rule, mx.cuh: scale 2^e, e = ceil(log2(amax / 448)),
// values rounded to nearest E4M3; with two terms the residual x - hi gets its
// own scales).  The value quantised is the one the quantiser pass sees, the sum
// of the BF16 hi and lo of the FP32 component (hi_lo_value), so both ways give
// the same bytes.  The row layout is the quantiser's: hi components at
// [0, Kq_pad), lo at [Kq_pad, 2 Kq_pad).

// bf16(x) + bf16(x - bf16(x)) in FP32: the component as its BF16 hi + lo pair holds it.
__device__ __forceinline__ float hi_lo_value(float x) {
  const float h = bf16_value(bf16_bits(x));
  return h + bf16_value(bf16_bits(x - h));
}

// Row r's components [c0, Kq_pad) past the tiles: zero E4M3 bytes, hi and (split)
// lo, and unit scales (c0 a multiple of 32).
__device__ __forceinline__ void mx_zero_tail(const MxQuantSide& q, int64_t r, int64_t c0) {
  uint8_t* row = q.dst + r * q.dst_pitch;
  for (int64_t c = c0; c < q.Kq_pad; c += 16) {
    *reinterpret_cast<uint4*>(row + c) = make_uint4(0u, 0u, 0u, 0u);
    if (q.qsplit > 1) *reinterpret_cast<uint4*>(row + q.Kq_pad + c) = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int64_t cg = c0 / 32; cg < q.Kq_pad / 32; ++cg) {
    q.sf[mx_sf_offset(q, r, cg)] = 127;
    if (q.qsplit > 1) q.sf[mx_sf_offset(q, r, q.Kq_pad / 32 + cg)] = 127;
  }
}

// Unit scales of runs [cg0, cg1) (hi, and lo with the split) for the rows
// [n_out, round_up(n_out, tile_rows)) that pad the last tile of scale blocks;
// the block's threads share the work.  Each tile of the last row of tiles takes
// its own runs, so no block does more than a few thousand bytes.
__device__ __forceinline__ void mx_pad_rows(const MxQuantSide& q, int64_t n_out, int64_t cg0, int64_t cg1) {
  const int64_t rows = (n_out + q.tile_rows - 1) / q.tile_rows * q.tile_rows - n_out;
  const int64_t kq = q.Kq_pad / 32;
  if (cg1 > kq) cg1 = kq;
  const int64_t nr = cg1 - cg0;
  if (rows <= 0 || nr <= 0) return;
  const int64_t total = rows * nr;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int64_t r = n_out + e / nr, cg = cg0 + e % nr;
    q.sf[mx_sf_offset(q, r, cg)] = 127;
    if (q.qsplit > 1) q.sf[mx_sf_offset(q, r, kq + cg)] = 127;
  }
}

// E4M3 of v[0..N) * inv (N = 1, 2, 4 or 8), packed two values a 16-bit half.
template <int N>
__device__ __forceinline__ void mx_quant(const float (&v)[N], float inv, uint32_t (&q)[N > 1 ? N / 2 : 1]) {
#pragma unroll
  for (int k = 0; k < (N > 1 ? N / 2 : 1); ++k) q[k] = e4m3x2(v[2 * k], N > 1 ? v[N > 1 ? 2 * k + 1 : 0] : 0.0f, inv);
}

// The N bytes at dst (aligned to N).
template <int N>
__device__ __forceinline__ void mx_put(uint8_t* dst, const uint32_t (&q)[N > 1 ? N / 2 : 1]) {
  if (N == 1) *dst = static_cast<uint8_t>(q[0] & 0xFFu);
  if (N == 2) *reinterpret_cast<uint16_t*>(dst) = static_cast<uint16_t>(q[0]);
  if (N == 4) *reinterpret_cast<uint32_t*>(dst) = q[0] | (q[N > 2 ? 1 : 0] << 16);
  if (N == 8)
    *reinterpret_cast<uint2*>(dst) =
        make_uint2(q[0] | (q[N > 2 ? 1 : 0] << 16), q[N > 4 ? 2 : 0] | (q[N > 4 ? 3 : 0] << 16));
}

// v - deq(q) 2^e, the residual of the values mx_quant rounded.
template <int N>
__device__ __forceinline__ void mx_residual(float (&v)[N], const uint32_t (&q)[N > 1 ? N / 2 : 1], float s) {
#pragma unroll
  for (int k = 0; k < (N > 1 ? N / 2 : 1); ++k) {
    const float2 d = e4m3x2_value(q[k]);
    v[2 * k] -= d.x * s;
    if (N > 1) v[N > 1 ? 2 * k + 1 : 0] -= d.y * s;
  }
}

// Rows, E4M3 (l+1 in {1, 2, 4, 8}): lane g holds the l+1 components of group g,
// so a run of 32 components is 32 / (l+1) neighbouring lanes; its amax is a
// butterfly over them and its first lane writes the scale byte.
template <typename InT, int LP1, bool kG, bool kBulk>
__device__ __forceinline__ void rows_tile_q(const TileCtx& c, const TileIn<InT, kBulk>& tin, const float* sCoef, int ux,
                                            int uy, const MxQuantSide& q) {
  constexpr int RL = 32 / LP1;   // lanes of one run
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gg = static_cast<int64_t>(ux) * 32 + lane;
  const int64_t comp0 = gg * LP1;
  const bool in_k = comp0 < q.Kq_pad;
  // (the batched form reads l+1 = 8 coefficients through L1 per use: 64 more live
  // registers would spill beside its job bookkeeping)
  const PtCoef<LP1, kG, !(kG && LP1 == 8)> cf(sCoef);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = static_cast<int64_t>(uy) * kPtBoxY + warp + 8 * u;
    float2 x[4];
    tin.group8(warp + 8 * u, lane, x);
    float v[LP1];
    float am = 0.0f;
#pragma unroll
    for (int p = 0; p < LP1; ++p) {
      v[p] = hi_lo_value(project_one(x, cf, p));
      am = fmaxf(am, fabsf(v[p]));
    }
    // every lane of the warp takes part in the butterflies (a row is live or not for all)
#pragma unroll
    for (int o = RL / 2; o >= 1; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    const int e = mx_exponent(am);
    uint32_t qw[LP1 > 1 ? LP1 / 2 : 1];
    mx_quant<LP1>(v, ldexpf(1.0f, -e), qw);
    const bool live = i < c.n_out && in_k;
    uint8_t* row = q.dst + (i < c.n_out ? i : 0) * q.dst_pitch;
    if (live) {
      mx_put<LP1>(row + comp0, qw);
      if (lane % RL == 0) q.sf[mx_sf_offset(q, i, comp0 / 32)] = static_cast<uint8_t>(e + 127);
    }
    if (q.qsplit > 1) {
      mx_residual<LP1>(v, qw, ldexpf(1.0f, e));
      float am2 = 0.0f;
#pragma unroll
      for (int p = 0; p < LP1; ++p) am2 = fmaxf(am2, fabsf(v[p]));
#pragma unroll
      for (int o = RL / 2; o >= 1; o >>= 1) am2 = fmaxf(am2, __shfl_xor_sync(0xffffffffu, am2, o));
      const int e2 = mx_exponent(am2);
      mx_quant<LP1>(v, ldexpf(1.0f, -e2), qw);
      if (live) {
        mx_put<LP1>(row + q.Kq_pad + comp0, qw);
        if (lane % RL == 0) q.sf[mx_sf_offset(q, i, q.Kq_pad / 32 + comp0 / 32)] = static_cast<uint8_t>(e2 + 127);
      }
    }
  }
  if (ux == c.units_x - 1 && lane == 0) {
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
      const int64_t i = static_cast<int64_t>(uy) * kPtBoxY + warp + 8 * u;
      if (i < c.n_out) mx_zero_tail(q, i, static_cast<int64_t>(c.units_x) * 32 * LP1);
    }
  }
  if (uy == c.units_y - 1) {   // padding rows: this tile's runs, and the last tile also the runs past the tiles
    const int64_t cg0 = static_cast<int64_t>(ux) * LP1;
    mx_pad_rows(q, c.n_out, cg0, ux == c.units_x - 1 ? q.Kq_pad / 32 : cg0 + LP1);
  }
}

// Columns, E4M3 (l+1 = 8): thread t's four groups of column t are exactly one
// run of 32 components of row j of B_d, quantised and written as 32 bytes.
template <typename InT, bool kG, bool kBulk>
__device__ __forceinline__ void cols_tile_q(const TileCtx& c, const TileIn<InT, kBulk>& tin, const float* sCoef, int ux,
                                            int uy, const MxQuantSide& q) {
  const int t = threadIdx.x;
  const int64_t j = static_cast<int64_t>(ux) * kPtBoxX + t;
  if (ux == c.units_x - 1)   // padding rows: this tile's run, and the last tile also the runs past the tiles
    mx_pad_rows(q, c.n_out, uy, uy == c.units_y - 1 ? q.Kq_pad / 32 : uy + 1);
  if (j >= c.n_out) return;
  const PtCoef<8, kG, false> cf(sCoef);
  float v[32];
  float am = 0.0f;
#pragma unroll
  for (int g4 = 0; g4 < 4; ++g4) {
    float2 x[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      x[e] = make_float2(tin.elem(g4 * 8 + 2 * e, t), tin.elem(g4 * 8 + 2 * e + 1, t));
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      v[g4 * 8 + p] = hi_lo_value(project_one(x, cf, p));
      am = fmaxf(am, fabsf(v[g4 * 8 + p]));
    }
  }
  uint8_t* row = q.dst + j * q.dst_pitch;
  const int64_t comp0 = static_cast<int64_t>(uy) * 32;
  if (comp0 < q.Kq_pad) {
    const int e = mx_exponent(am);
    const float inv = ldexpf(1.0f, -e);
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = e4m3x2(v[4 * k], v[4 * k + 1], inv) | (e4m3x2(v[4 * k + 2], v[4 * k + 3], inv) << 16);
    reinterpret_cast<uint4*>(row + comp0)[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<uint4*>(row + comp0)[1] = make_uint4(w[4], w[5], w[6], w[7]);
    q.sf[mx_sf_offset(q, j, uy)] = static_cast<uint8_t>(e + 127);
    if (q.qsplit > 1) {
      const float sc = ldexpf(1.0f, e);
      float am2 = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float2 a = e4m3x2_value(w[k] & 0xFFFFu), b = e4m3x2_value(w[k] >> 16);
        v[4 * k] -= a.x * sc;
        v[4 * k + 1] -= a.y * sc;
        v[4 * k + 2] -= b.x * sc;
        v[4 * k + 3] -= b.y * sc;
        am2 = fmaxf(am2, fmaxf(fmaxf(fabsf(v[4 * k]), fabsf(v[4 * k + 1])), fmaxf(fabsf(v[4 * k + 2]), fabsf(v[4 * k + 3]))));
      }
      const int e2 = mx_exponent(am2);
      const float inv2 = ldexpf(1.0f, -e2);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        w[k] = e4m3x2(v[4 * k], v[4 * k + 1], inv2) | (e4m3x2(v[4 * k + 2], v[4 * k + 3], inv2) << 16);
      reinterpret_cast<uint4*>(row + q.Kq_pad + comp0)[0] = make_uint4(w[0], w[1], w[2], w[3]);
      reinterpret_cast<uint4*>(row + q.Kq_pad + comp0)[1] = make_uint4(w[4], w[5], w[6], w[7]);
      q.sf[mx_sf_offset(q, j, q.Kq_pad / 32 + uy)] = static_cast<uint8_t>(e2 + 127);
    }
  }
  if (uy == c.units_y - 1) mx_zero_tail(q, j, static_cast<int64_t>(c.units_y) * 32);
}

// The packed lead hi and lo terms of four whole groups (tiered split, tl <= 2).
__device__ __forceinline__ void store_lead_runs(const TileCtx& c, uint16_t* orow, int64_t g0, const uint32_t (&lh)[4],
                                                const uint32_t (&ll)[4]) {
  uint16_t* lhp = orow + c.Kp_pad + g0 * c.tl;
  uint16_t* llp = orow + c.Kp_pad + c.Kt_pad + g0 * c.tl;
  if (c.tl == 1) {
    *reinterpret_cast<uint2*>(lhp) = make_uint2(lh[0], lh[1]);
    *reinterpret_cast<uint2*>(llp) = make_uint2(ll[0], ll[1]);
  } else {
    *reinterpret_cast<uint4*>(lhp) = make_uint4(lh[0], lh[1], lh[2], lh[3]);
    *reinterpret_cast<uint4*>(llp) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
  }
}

// Cols: tile = 32 rows of B (4 groups) x 256 columns.  Thread t owns column
// t of the tile and writes its 4 (l+1) components contiguously into row j of
// B_d (the transposed, K-major layout the GEMM reads); for l+1 <= 2 the four
// groups' components are packed into one 8- or 16-byte store.  For FP32 input
// with l+1 = 4 or 8 and four whole groups, the warp stages its runs in its own
// 128-byte column slice of the tile (read completely before it is
// overwritten) and writes them row by row (run_put_group / runs_write).
template <typename InT, int LP1, bool kG, bool kTiered>
__device__ __forceinline__ void cols_tile(const TileCtx& c, const TileIn<InT, false>& tin, const float* sCoef, int ux,
                                          int uy) {
  constexpr int row_bytes = TileIn<InT, false>::kRowBytes;
  const int t = threadIdx.x;
  const int64_t j = static_cast<int64_t>(ux) * kPtBoxX + t;
  const int64_t g0 = static_cast<int64_t>(uy) * 4;
  const bool full = g0 + 4 <= c.NG;
  constexpr bool tiered = kTiered;
  constexpr bool kStaged = sizeof(InT) == 4 && (LP1 == 4 || LP1 == 8);
  const PtCoef<LP1, kG, (LP1 <= 4)> cf(sCoef);
  const bool need_lo = c.nsplit > 1;   // (the tiered lead terms are split as well)
  if constexpr (kStaged) {
    if (full) {
      // every lane of the warp takes part (columns past the output are zeros of
      // the TMA fill and are not written back)
      const int lane = t & 31, w = t >> 5;
      uint8_t* base = tin.base + w * 128;
      const bool two = !tiered && c.nsplit > 1;
      uint32_t lh[4] = {0u, 0u, 0u, 0u}, ll[4] = {0u, 0u, 0u, 0u};  // packed lead runs for tl <= 2
      float x[32];
  #pragma unroll
      for (int e = 0; e < 32; ++e) x[e] = tin.elem(e, t);
      __syncwarp();  // the warp's column slice is read; it now takes the staged runs
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 xq[4];
  #pragma unroll
        for (int e = 0; e < 4; ++e) xq[e] = make_float2(x[q * 8 + 2 * e], x[q * 8 + 2 * e + 1]);
        uint16_t hi[8], lo[8];
        project8(xq, cf, need_lo, hi, lo);
        run_put_group<LP1>(base, row_bytes, 0, lane, q, hi);
        if (two) run_put_group<LP1>(base, row_bytes, 1, lane, q, lo);
        if (tiered) {
          if (c.tl == 1) {
            lh[q >> 1] |= uint32_t(hi[0]) << (16 * (q & 1));
            ll[q >> 1] |= uint32_t(lo[0]) << (16 * (q & 1));
          } else if (c.tl == 2) {
            lh[q] = pack2(hi[0], hi[1]);
            ll[q] = pack2(lo[0], lo[1]);
          } else if (j < c.n_out) {
            uint16_t* orow = c.out + j * c.pitch;
            store_upto8(orow + c.Kp_pad + (g0 + q) * c.tl, hi, c.tl);
            store_upto8(orow + c.Kp_pad + c.Kt_pad + (g0 + q) * c.tl, lo, c.tl);
          }
        }
      }
      if (tiered && c.tl <= 2 && j < c.n_out) store_lead_runs(c, c.out + j * c.pitch, g0, lh, ll);
      __syncwarp();
      const int64_t jw = static_cast<int64_t>(ux) * kPtBoxX + w * 32;
      const int ncols = c.n_out - jw < 32 ? static_cast<int>(c.n_out - jw) : 32;
      uint16_t* o0 = c.out + jw * c.pitch + g0 * LP1;
      runs_write<LP1>(base, row_bytes, 0, lane, o0, c.pitch, ncols);
      if (two) runs_write<LP1>(base, row_bytes, 1, lane, o0 + c.Kp_pad, c.pitch, ncols);
      // the staging writes must be ordered before the next TMA fill of this stage
      fence_proxy_async_smem();
      if (uy == c.units_y - 1 && j < c.n_out) zero_row_tails(c, c.out + j * c.pitch, LP1);
      return;
    }
  }
  if (j >= c.n_out) return;
  uint16_t* orow = c.out + j * c.pitch;
  uint16_t* o = orow + g0 * LP1;
  uint32_t ph[4] = {0u, 0u, 0u, 0u}, pl[4] = {0u, 0u, 0u, 0u};  // packed runs for l+1 <= 2
  uint32_t lh[4] = {0u, 0u, 0u, 0u}, ll[4] = {0u, 0u, 0u, 0u};  // packed lead runs for tl <= 2
  // l+1 in {3, 5, 6, 7}, four whole groups: the 4 (l+1) components packed into words,
  // stored as (l+1) 8-byte chunks (the run starts 8 (l+1) uy bytes into the row)
  constexpr int kW = kOddRun<LP1> ? 2 * LP1 : 1;
  uint32_t wh[kW], wl[kW];
#pragma unroll
  for (int k = 0; k < kW; ++k) wh[k] = wl[k] = 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 x[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      x[e] = make_float2(tin.elem(q * 8 + 2 * e, t), tin.elem(q * 8 + 2 * e + 1, t));
    uint16_t hi[8], lo[8];
    project8(x, cf, need_lo, hi, lo);
    if (LP1 == 1) {
      ph[q >> 1] |= uint32_t(hi[0]) << (16 * (q & 1));
      pl[q >> 1] |= uint32_t(lo[0]) << (16 * (q & 1));
    } else if (LP1 == 2) {
      ph[q] = pack2(hi[0], hi[1]);
      pl[q] = pack2(lo[0], lo[1]);
    }
    if (kOddRun<LP1> && full) {
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        if (p >= LP1) break;
        const int e = (q * LP1 + p) % (2 * kW);   // (the modulus only keeps non-odd l+1 in range)
        wh[(e >> 1) % kW] |= uint32_t(hi[p]) << (16 * (e & 1));
        wl[(e >> 1) % kW] |= uint32_t(lo[p]) << (16 * (e & 1));
      }
    } else if ((LP1 > 2 || !full) && g0 + q < c.NG) {
      store_upto8(o + q * LP1, hi, LP1);
      if (!tiered && c.nsplit > 1) store_upto8(o + c.Kp_pad + q * LP1, lo, LP1);
    }
    if (tiered) {
      // the lead terms of the four groups are contiguous in their segments:
      // packed like the l+1 <= 2 runs when tl <= 2, one run per group otherwise
      if (c.tl == 1) {
        lh[q >> 1] |= uint32_t(hi[0]) << (16 * (q & 1));
        ll[q >> 1] |= uint32_t(lo[0]) << (16 * (q & 1));
      } else if (c.tl == 2) {
        lh[q] = pack2(hi[0], hi[1]);
        ll[q] = pack2(lo[0], lo[1]);
      }
      if ((c.tl > 2 || !full) && g0 + q < c.NG) {
        store_upto8(orow + c.Kp_pad + (g0 + q) * c.tl, hi, c.tl);
        store_upto8(orow + c.Kp_pad + c.Kt_pad + (g0 + q) * c.tl, lo, c.tl);
      }
    }
  }
  if (kOddRun<LP1> && full) {
#pragma unroll
    for (int k = 0; k < kW / 2; ++k) reinterpret_cast<uint2*>(o)[k] = make_uint2(wh[2 * k], wh[2 * k + 1]);
    if (!tiered && c.nsplit > 1)
#pragma unroll
      for (int k = 0; k < kW / 2; ++k)
        reinterpret_cast<uint2*>(o + c.Kp_pad)[k] = make_uint2(wl[2 * k], wl[2 * k + 1]);
  }
  if (full && LP1 == 1) {
    *reinterpret_cast<uint2*>(o) = make_uint2(ph[0], ph[1]);
    if (c.nsplit > 1 && !tiered) *reinterpret_cast<uint2*>(o + c.Kp_pad) = make_uint2(pl[0], pl[1]);
  } else if (full && LP1 == 2) {
    *reinterpret_cast<uint4*>(o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    if (c.nsplit > 1 && !tiered) *reinterpret_cast<uint4*>(o + c.Kp_pad) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
  }
  if (tiered && full && c.tl <= 2) store_lead_runs(c, orow, g0, lh, ll);
  if (uy == c.units_y - 1) zero_row_tails(c, orow, LP1);
}

// The ring of one block: NST tile buffers with a full and an empty barrier
// each (PtStages).  Thread 0 issues the
// copies: the first NST up front, and then each refill right after its own
// warp has finished the tile it replaces (it waits for the other warps to
// finish that tile as well, so it never waits on itself).  Tile k of the block
// uses stage k % NST in phase (k / NST) & 1 of both barriers.
struct PtRing {
  uint64_t* full;
  uint64_t* empty;
  int64_t issued = 0;   // copies issued (thread 0 only)
};

// FP32: three 32 KB stages, two blocks per SM.  BF16: four 16 KB stages, so
// three blocks fit an SM (24 warps to hide the projection's dependent
// arithmetic; 192 KB in flight per SM either way).  Bulk tiles take 16 bytes
// more per row.
template <typename InT, bool kBulk = false>
struct PtStages {
  static constexpr int kBytes = kPtBoxY * TileIn<InT, kBulk>::kRowBytes;
  static constexpr int kCount = sizeof(InT) == 4 ? kPtStages : 4;
  static constexpr int kRing = kCount * kBytes;
  static constexpr int kSmem = 1024 + kRing + 1024;
};
static_assert(PtStages<float>::kRing <= kPtStages * kPtTileMax &&
                  PtStages<__nv_bfloat16>::kRing <= kPtStages * kPtTileMax,
              "rings fit the FP32 budget");
static_assert(2 * (PtStages<float, true>::kSmem + 1024) <= 228 * 1024 &&
                  3 * (PtStages<__nv_bfloat16, true>::kSmem + 1024) <= 228 * 1024,
              "bulk rings keep the blocks per SM");

// Thread 0: waits until tile k (the stage's previous user) is released, then
// the caller issues the copy of tile k + NST.  k < 0: the stage is fresh.
template <int NST>
__device__ __forceinline__ bool pt_stage_free(const PtRing& r, int64_t k, int* err) {
  if (k < 0) return true;
  const int s = static_cast<int>(k % NST);
  return mbar_wait(&r.empty[s], static_cast<uint32_t>((k / NST) & 1), err, DEV_TIMEOUT_EMPTY);
}

// Thread 0, after the loop: every issued copy must land before the block exits
// (copies past the last consumed tile exist only after a timeout).
template <int NST>
__device__ __forceinline__ void pt_drain(const PtRing& r, int64_t consumed, int* err) {
  for (int64_t k = consumed; k < r.issued; ++k)
    if (!mbar_wait_drain(&r.full[k % NST], static_cast<uint32_t>((k / NST) & 1)))
      atomicCAS(err, 0, DEV_TIMEOUT_DRAIN);
}

template <typename InT, int LP1, bool kTiered, bool kQ>
// 256 threads and at most 128 registers: two blocks fit an SM (four warps of
// each block per scheduler, 4 x 32 x 128 = 16 K registers), and the l+1 = 8
// paths need no spills.
__global__ void __launch_bounds__(kPtThreads, 2) project_tma_kernel(const __grid_constant__ ProjTmaParams p) {
  constexpr int NST = PtStages<InT>::kCount, TB = PtStages<InT>::kBytes;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* tiles = sm;
  // After the tiles: 2 x NST mbarriers at +0; the 8 x (l+1) basis
  // values of each side at +256 and +512 (8-byte aligned for the coefficient
  // pairs); at +768 the (side, tile column, tile row) of each stage's tile,
  // written by thread 0 when it issues the copy (so no consumer divides).
  PtRing ring{reinterpret_cast<uint64_t*>(sm + PtStages<InT>::kRing),
              reinterpret_cast<uint64_t*>(sm + PtStages<InT>::kRing) + NST};
  float* sCoef = reinterpret_cast<float*>(sm + PtStages<InT>::kRing + 256);
  int4* stage_unit = reinterpret_cast<int4*>(sm + PtStages<InT>::kRing + 768);
  static_assert(NST * TB == PtStages<InT>::kRing && 2 * NST * 8 <= 256 && 768 + NST * 16 <= 1024,
                "layout of the block's control area");
  const int lane = threadIdx.x & 31;
  const int64_t n0 = p.side[0].num_units, total = n0 + p.side[1].num_units;
  const int64_t mine = blockIdx.x < total ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&ring.full[s], 1);
      mbar_init(&ring.empty[s], kPtConsumers / 32);
    }
    fence_mbar_init();
  }
  if (threadIdx.x < 128) {
    // Stage the kept basis vectors of side sd as sCoef[sd * 64 + q * 8 + t].
    const int sd = threadIdx.x >> 6, k = threadIdx.x & 63, q = k >> 3, t = k & 7;
    if (q < LP1 && p.side[sd].num_units > 0)
      sCoef[threadIdx.x] = sd == 0 ? p.side[0].coef[t * LP1 + q] : p.side[1].coef[q * 8 + t];
  }
  __syncthreads();

  // Thread 0 issues the copy of the block's tile k into stage k % NST.
  auto issue = [&](int64_t k) {
    const int64_t u = blockIdx.x + k * gridDim.x;
    const int s = static_cast<int>(k % NST);
    const int sd = u >= n0 ? 1 : 0;
    const ProjSide& S = p.side[sd];
    const int64_t v = u - (sd ? n0 : 0);
    const int ux = static_cast<int>(v % S.units_x), uy = static_cast<int>(v / S.units_x);
    stage_unit[s] = make_int4(sd, ux, uy, 0);
    mbar_arrive_expect_tx(&ring.full[s], static_cast<uint32_t>(S.tile_bytes));
    tma_load_2d(tiles + s * TB, &p.map[sd], &ring.full[s], ux * kPtBoxX, uy * kPtBoxY);
    ring.issued = k + 1;
  };
  if (threadIdx.x == 0) {
    if (p.side[0].num_units > 0) tma_prefetch(&p.map[0]);
    if (p.side[1].num_units > 0) tma_prefetch(&p.map[1]);
    for (int64_t k = 0; k < NST && k < mine; ++k) issue(k);
  }

  int64_t k = 0;
  for (; k < mine; ++k) {
    const int s = static_cast<int>(k % NST);
    if (!mbar_wait(&ring.full[s], static_cast<uint32_t>((k / NST) & 1), p.err, DEV_TIMEOUT_FULL)) break;
    const TileIn<InT, false> tin{tiles + s * TB, 0, 0, kPtBoxY, kPtBoxX};
    const int4 un = stage_unit[s];
    const int sd = un.x, ux = un.y, uy = un.z;
    const ProjSide& S = p.side[sd];
    const TileCtx c{S.out, S.n_out, p.NG, p.pitch, p.Kp_pad, p.Kt_pad, S.units_x, S.units_y, p.nsplit, p.tl};
    if (sd == 0) {
      if constexpr (kQ)
        rows_tile_q<InT, LP1, false, false>(c, tin, sCoef, ux, uy, p.q[0]);
      else
        rows_tile<InT, LP1, false, kTiered>(c, tin, sCoef, ux, uy);
    } else {
      if constexpr (kQ) {
        if constexpr (LP1 == 8) cols_tile_q<InT, false, false>(c, tin, sCoef + 64, ux, uy, p.q[1]);
      } else {
        cols_tile<InT, LP1, false, kTiered>(c, tin, sCoef + 64, ux, uy);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&ring.empty[s]);
    if (threadIdx.x == 0 && k + NST < mine) {
      if (!pt_stage_free<NST>(ring, k, p.err)) {
        ++k;
        break;
      }
      issue(k + NST);
    }
  }
  if (threadIdx.x == 0) pt_drain<NST>(ring, k, p.err);
}

// Batched form: units of many operands, each tile's job read from a unit
// list; the consumers take the job and tile coordinates from the stage they
// wait on, and read the job's coefficients through the L1 cache.  TMA jobs
// (units int4 {job, ux, uy, 0}): thread 0 issues each tile as one tensor copy.
// Bulk jobs (kBulk: operands whose row pitch or base TMA cannot address; units
// of two int4, {job, ux, uy, bulk_tile_word} and the address of the tile's
// first element and the row pitch in bytes, 64-bit each): warp 0 issues them,
// lane r copying tile row r from the 16-byte granule that holds its first
// element to the one that holds its last (inside the granules of the operand's
// own first and last bytes, which never cross a page), after lane 0 has
// announced the tile's total bytes on the stage's barrier.  Bulk tiles are read
// by the E4M3 projections only: with BF16 output (whose column path stages its
// runs in the tile, where the shifted rows of the neighbouring warps lie) they
// measured slower than the per-group job kernels.
template <typename InT, int LP1, bool kQ, bool kBulk>
__global__ void __launch_bounds__(kPtThreads, 2) project_tma_jobs_kernel(const TmaJob* __restrict__ jobs,
                                                                           const int4* __restrict__ units,
                                                                           int64_t total, int* err) {
  static_assert(kQ || !kBulk, "bulk tiles feed the E4M3 projections");
  using St = PtStages<InT, kBulk>;
  using Tin = TileIn<InT, kBulk>;
  constexpr int NST = St::kCount, TB = St::kBytes;
  constexpr int ES = static_cast<int>(sizeof(InT));
  constexpr int UW = kBulk ? 2 : 1;   // int4 per unit
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* tiles = sm;
  PtRing ring{reinterpret_cast<uint64_t*>(sm + St::kRing), reinterpret_cast<uint64_t*>(sm + St::kRing) + NST};
  int4* stage_unit = reinterpret_cast<int4*>(sm + St::kRing + 256);
  static_assert(NST * TB == St::kRing && 2 * NST * 8 <= 256 && 256 + NST * 16 <= 1024,
                "layout of the block's control area");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = kBulk ? warp == 0 : threadIdx.x == 0;
  const int64_t mine = blockIdx.x < total ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&ring.full[s], 1);
      mbar_init(&ring.empty[s], kPtConsumers / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();

  auto fetch = [&](int64_t k, int4& u0, int4& u1) {
    const int64_t u = (blockIdx.x + k * gridDim.x) * UW;
    u0 = __ldg(units + u);
    if (kBulk) u1 = __ldg(units + u + 1);
  };
  // Issues tile k (unit u0, u1) into its stage: thread 0 (TMA) or warp 0 (bulk).
  auto issue = [&](int64_t k, const int4& u0, const int4& u1) {
    const int s = static_cast<int>(k % NST);
    if constexpr (kBulk) {
      const int nrows = (u0.w >> 8) & 0xff, nx = (u0.w >> 16) & 0x1ff;
      const uint64_t row0 = static_cast<uint32_t>(u1.x) | (static_cast<uint64_t>(static_cast<uint32_t>(u1.y)) << 32);
      const uint64_t ldb = static_cast<uint32_t>(u1.z) | (static_cast<uint64_t>(static_cast<uint32_t>(u1.w)) << 32);
      const bool live = lane < nrows;
      const uint64_t a = row0 + static_cast<uint64_t>(live ? lane : 0) * ldb;
      const uint64_t lo = a & ~uint64_t(15), hi = (a + static_cast<uint64_t>(nx) * ES + 15) & ~uint64_t(15);
      const uint32_t bytes = live ? static_cast<uint32_t>(hi - lo) : 0u;
      const uint32_t sum = __reduce_add_sync(0xffffffffu, bytes);
      if (lane == 0) {
        stage_unit[s] = u0;
        mbar_arrive_expect_tx(&ring.full[s], sum);
      }
      __syncwarp();
      if (live) bulk_load(tiles + s * TB + lane * Tin::kRowBytes, reinterpret_cast<const void*>(lo), bytes, &ring.full[s]);
    } else {
      stage_unit[s] = u0;
      mbar_arrive_expect_tx(&ring.full[s], static_cast<uint32_t>(TB));
      tma_load_2d(tiles + s * TB, &jobs[u0.x].map, &ring.full[s], u0.y * kPtBoxX, u0.z * kPtBoxY);
    }
    ring.issued = k + 1;
  };
  if (producer)
    for (int64_t k = 0; k < NST && k < mine; ++k) {
      int4 u0, u1 = make_int4(0, 0, 0, 0);
      fetch(k, u0, u1);
      issue(k, u0, u1);
    }

  int64_t k = 0;
  for (; k < mine; ++k) {
    const int s = static_cast<int>(k % NST);
    if (!mbar_wait(&ring.full[s], static_cast<uint32_t>((k / NST) & 1), err, DEV_TIMEOUT_FULL)) break;
    const int4 un = stage_unit[s];
    const TmaJob& J = jobs[un.x];
    const TileCtx c{J.out, J.n_out, J.NG, J.pitch, J.Kp_pad, J.Kt_pad, J.units_x, J.units_y, J.nsplit, J.tl};
    // bulk tile word: a0 | ldm << 4 | rows << 8 | cols << 16
    const Tin tin{tiles + s * TB, un.w & 15, (un.w >> 4) & 15, kBulk ? (un.w >> 8) & 0xff : kPtBoxY,
                  kBulk ? (un.w >> 16) & 0x1ff : kPtBoxX};
    if constexpr (kQ) {   // E4M3 output (J.q): rows with l+1 in {1, 2, 4, 8}, columns with l+1 = 8
      if (J.cols) {
        if constexpr (LP1 == 8) cols_tile_q<InT, true, kBulk>(c, tin, J.coef, un.y, un.z, J.q);
      } else {
        rows_tile_q<InT, LP1, true, kBulk>(c, tin, J.coef, un.y, un.z, J.q);
      }
    } else if constexpr (!kBulk) {
      if (J.cols)
        cols_tile<InT, LP1, true, false>(c, tin, J.coef, un.y, un.z);
      else
        rows_tile<InT, LP1, true, false>(c, tin, J.coef, un.y, un.z);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&ring.empty[s]);
    if (producer && k + NST < mine) {
      bool ok = threadIdx.x == 0 ? pt_stage_free<NST>(ring, k, err) : true;
      if (kBulk) ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        ++k;
        break;
      }
      int4 u0, u1 = make_int4(0, 0, 0, 0);
      fetch(k + NST, u0, u1);
      issue(k + NST, u0, u1);
    }
  }
  if (threadIdx.x == 0) pt_drain<NST>(ring, k, err);
}

bool make_input_map(CUtensorMap* map, const void* base, int in_dtype, int64_t inner, int64_t rows, int64_t ld) {
  const size_t es = in_dtype == PJ_BF16 ? 2 : 4;
  const uint64_t dims[2] = {static_cast<uint64_t>(inner), static_cast<uint64_t>(rows)};
  const uint64_t strides[1] = {static_cast<uint64_t>(ld) * es};
  const uint32_t box[2] = {kPtBoxX, kPtBoxY};
  return make_tmap_plain_load(map, in_dtype == PJ_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              base, 2, dims, strides, box);
}

bool tma_shape_ok(const void* base, int in_dtype, int64_t inner, int64_t rows, int64_t ld) {
  const size_t es = in_dtype == PJ_BF16 ? 2 : 4;
  return (reinterpret_cast<uintptr_t>(base) % 16 == 0) && ((ld * es) % 16 == 0) && inner >= kPtBoxX &&
         rows >= kPtBoxY && inner < (int64_t(1) << 31) && rows < (int64_t(1) << 31) && ld >= inner;
}

// One instantiation per input dtype and l+1 (1..8), so the projection loops
// carry no predicated-off work.
using TmaKernel = void (*)(ProjTmaParams);

// A tiered split (lead projections only carry the lo term) has its own
// instantiations, so the plain path keeps its register budget.
template <typename InT, bool kTiered>
TmaKernel tma_kernel_for(int lp1) {
  switch (lp1) {
    case 1: return project_tma_kernel<InT, 1, kTiered, false>;
    case 2: return project_tma_kernel<InT, 2, kTiered, false>;
    case 3: return project_tma_kernel<InT, 3, kTiered, false>;
    case 4: return project_tma_kernel<InT, 4, kTiered, false>;
    case 5: return project_tma_kernel<InT, 5, kTiered, false>;
    case 6: return project_tma_kernel<InT, 6, kTiered, false>;
    case 7: return project_tma_kernel<InT, 7, kTiered, false>;
    default: return project_tma_kernel<InT, 8, kTiered, false>;
  }
}

// E4M3 output (l+1 in {1, 2, 4, 8}; columns only with l+1 = 8).
template <typename InT>
TmaKernel tma_q_kernel_for(int lp1) {
  switch (lp1) {
    case 1: return project_tma_kernel<InT, 1, false, true>;
    case 2: return project_tma_kernel<InT, 2, false, true>;
    case 4: return project_tma_kernel<InT, 4, false, true>;
    default: return project_tma_kernel<InT, 8, false, true>;
  }
}

cudaError_t launch_tma(const ProjTmaParams& p, int in_dtype, int lp1, int sms, cudaStream_t st, bool quant = false) {
  // The shared-memory opt-in is recorded per device and kernel; repeating it
  // from a racing thread is harmless.
  // The shared-memory opt-in and the blocks per SM are recorded per device and
  // kernel (0: not yet); repeating them from a racing thread is harmless.
  static int blocks_per_sm[2][2][2][8][64] = {};
  const int which = in_dtype == PJ_BF16 ? 1 : 0;
  const int smem = which ? PtStages<__nv_bfloat16>::kSmem : PtStages<float>::kSmem;
  const int tiered = p.nsplit > 1 && p.tl < lp1 ? 1 : 0;
  const int li = lp1 - 1;
  TmaKernel kern = which ? (tiered ? tma_kernel_for<__nv_bfloat16, true>(lp1) : tma_kernel_for<__nv_bfloat16, false>(lp1))
                         : (tiered ? tma_kernel_for<float, true>(lp1) : tma_kernel_for<float, false>(lp1));
  if (quant) kern = which ? tma_q_kernel_for<__nv_bfloat16>(lp1) : tma_q_kernel_for<float>(lp1);
  const int qi = quant ? 1 : 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nb = dev >= 0 && dev < 64 ? blocks_per_sm[qi][which][tiered][li][dev] : 0;
  if (nb == 0) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kPtThreads, smem);
    if (e != cudaSuccess) return e;
    nb = nb < 1 ? 1 : nb;
    if (dev >= 0 && dev < 64) blocks_per_sm[qi][which][tiered][li][dev] = nb;
  }
  const int64_t units = p.side[0].num_units + p.side[1].num_units;
  const int64_t slots = static_cast<int64_t>(nb) * sms;
  const int64_t grid = units < slots ? units : slots;
  kern<<<static_cast<unsigned>(grid), kPtThreads, smem, st>>>(p);
  return cudaGetLastError();
}

// Fills side sd of p when the operand suits TMA; returns whether it does.
bool tma_side(ProjTmaParams& p, int sd, const void* X, int64_t ld, int in_dtype, int64_t inner, int64_t rows,
              int64_t n_out, const float* coef, uint16_t* out) {
  if (!X || n_out == 0 || !tma_shape_ok(X, in_dtype, inner, rows, ld)) return false;
  if (!make_input_map(&p.map[sd], X, in_dtype, inner, rows, ld)) return false;
  ProjSide& S = p.side[sd];
  S.coef = coef;
  S.out = out;
  S.n_out = n_out;
  S.units_x = static_cast<int>(ceil_div(inner, kPtBoxX));
  S.units_y = static_cast<int>(ceil_div(rows, kPtBoxY));
  S.num_units = static_cast<int64_t>(S.units_x) * S.units_y;
  S.tile_bytes = kPtBoxX * kPtBoxY * (in_dtype == PJ_BF16 ? 2 : 4);
  return true;
}

}  // namespace

cudaError_t launch_project_pair_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int in_dtype,
                                     const GemmGeom& g, const float* Cs, const float* Ds, uint16_t* Ac,
                                     uint16_t* Bd, int* err, int sms, cudaStream_t st) {
  if (g.K == 0) return cudaSuccess;
  if (g.M == 0) A = nullptr;
  if (g.N == 0) B = nullptr;
  bool rows_tma = false, cols_tma = false;
  if (g.L == 8 && g.lp1 >= 1 && g.lp1 <= 8) {
    ProjTmaParams p{};
    p.pitch = gemm_pitch(g);
    p.Kp_pad = g.Kp_pad;
    p.Kt_pad = g.Kt_pad;
    p.NG = ceil_div(g.K, 8);
    p.nsplit = g.nsplit;
    p.tl = g.tl;
    p.err = err;
    rows_tma = tma_side(p, 0, A, lda, in_dtype, g.K, g.M, g.M, Cs, Ac);
    cols_tma = tma_side(p, 1, B, ldb, in_dtype, g.N, g.K, g.N, Ds, Bd);
    if (rows_tma || cols_tma) {
      const cudaError_t e = launch_tma(p, in_dtype, g.lp1, sms, st);
      if (e != cudaSuccess) return e;
    }
  }
  if (A && !rows_tma) {
    const cudaError_t e = launch_project_rows_simt(A, lda, in_dtype, g, Cs, Ac, st);
    if (e != cudaSuccess) return e;
  }
  if (B && !cols_tma) return launch_project_cols_simt(B, ldb, in_dtype, g, Ds, Bd, st);
  return cudaSuccess;
}

bool project_mx_fusable(const GemmGeom& g, int side) {
  if (g.L != 8 || (g.nsplit > 1 && g.tl < g.lp1)) return false;
  return side == 0 ? (g.lp1 == 1 || g.lp1 == 2 || g.lp1 == 4 || g.lp1 == 8) : g.lp1 == 8;
}

cudaError_t launch_project_pair_mx(const void* A, int64_t lda, const void* B, int64_t ldb, int in_dtype,
                                   const GemmGeom& g, const float* Cs, const float* Ds, const MxQuantSide* qa,
                                   const MxQuantSide* qb, int* err, int sms, cudaStream_t st, bool* a_done,
                                   bool* b_done) {
  *a_done = *b_done = false;
  if (g.K == 0) return cudaSuccess;
  if (g.M == 0) A = nullptr;
  if (g.N == 0) B = nullptr;
  ProjTmaParams p{};
  p.pitch = gemm_pitch(g);
  p.Kp_pad = g.Kp_pad;
  p.Kt_pad = g.Kt_pad;
  p.NG = ceil_div(g.K, 8);
  p.nsplit = g.nsplit;
  p.tl = g.tl;
  p.err = err;
  if (A && qa && project_mx_fusable(g, 0) && tma_side(p, 0, A, lda, in_dtype, g.K, g.M, g.M, Cs, nullptr)) {
    p.q[0] = *qa;
    *a_done = true;
  }
  if (B && qb && project_mx_fusable(g, 1) && tma_side(p, 1, B, ldb, in_dtype, g.N, g.K, g.N, Ds, nullptr)) {
    p.q[1] = *qb;
    *b_done = true;
  }
  // With both operands given and only one side suited, both take the BF16 pass: one
  // projection launch for both and the quantiser measured faster than two launches.
  if (A && B && *a_done != *b_done) *a_done = *b_done = false;
  if (!*a_done) p.side[0].num_units = 0;
  if (!*b_done) p.side[1].num_units = 0;
  if (!*a_done && !*b_done) return cudaSuccess;
  return launch_tma(p, in_dtype, g.lp1, sms, st, true);
}

cudaError_t launch_project_rows_bf16(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs,
                                     uint16_t* Ac, int* err, int sms, cudaStream_t st) {
  return launch_project_pair_bf16(A, lda, nullptr, 0, in_dtype, g, Cs, nullptr, Ac, nullptr, err, sms, st);
}

cudaError_t launch_project_cols_bf16(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds,
                                     uint16_t* Bd, int* err, int sms, cudaStream_t st) {
  return launch_project_pair_bf16(nullptr, 0, B, ldb, in_dtype, g, nullptr, Ds, nullptr, Bd, err, sms, st);
}

bool tma_projection_ok(const void* X, int in_dtype, int64_t inner, int64_t rows, int64_t ld) {
  return X && tma_shape_ok(X, in_dtype, inner, rows, ld);
}

void bulk_job_units(const TmaJob& J, int in_dtype, int job, std::vector<int4>& out) {
  const int64_t es = in_dtype == PJ_BF16 ? 2 : 4;
  const uint64_t ldb = static_cast<uint64_t>(J.ld) * es;
  for (int uy = 0; uy < J.units_y; ++uy)
    for (int ux = 0; ux < J.units_x; ++ux) {
      const int64_t x0 = static_cast<int64_t>(ux) * kPtBoxX, y0 = static_cast<int64_t>(uy) * kPtBoxY;
      const int nx = static_cast<int>(J.inner - x0 < kPtBoxX ? J.inner - x0 : kPtBoxX);
      const int nrows = static_cast<int>(J.rows - y0 < kPtBoxY ? J.rows - y0 : kPtBoxY);
      const uint64_t row0 = reinterpret_cast<uint64_t>(J.src) + static_cast<uint64_t>(y0 * J.ld + x0) * es;
      const int word = static_cast<int>(row0 & 15) | static_cast<int>((ldb & 15) << 4) | (nrows << 8) | (nx << 16);
      out.push_back(make_int4(job, ux, uy, word));
      out.push_back(make_int4(static_cast<int>(row0 & 0xffffffffu), static_cast<int>(row0 >> 32),
                              static_cast<int>(ldb & 0xffffffffu), static_cast<int>(ldb >> 32)));
    }
}

bool bulk_projection_ok(const void* X, int in_dtype, int64_t inner, int64_t rows, int64_t ld) {
  const size_t es = in_dtype == PJ_BF16 ? 2 : 4;
  return X && reinterpret_cast<uintptr_t>(X) % es == 0 && inner >= 1 && rows >= 1 && ld >= inner &&
         inner < (int64_t(1) << 31) && rows < (int64_t(1) << 31);
}

void tma_job_grid(const GemmGeom& g, int cols, int* units_x, int* units_y) {
  const int64_t inner = cols ? g.N : g.K, rows = cols ? g.K : g.M;
  *units_x = static_cast<int>(ceil_div(inner, kPtBoxX));
  *units_y = static_cast<int>(ceil_div(rows, kPtBoxY));
}

int64_t tma_job_units(const GemmGeom& g, int cols) {
  int ux = 0, uy = 0;
  tma_job_grid(g, cols, &ux, &uy);
  return static_cast<int64_t>(ux) * uy;
}

bool make_tma_job(const void* X, int64_t ld, int in_dtype, int cols, const GemmGeom& g, const float* coef,
                  uint16_t* out, TmaJob* J, const MxQuantSide* q, bool bulk) {
  memset(J, 0, sizeof(TmaJob));
  const int64_t inner = cols ? g.N : g.K, rows = cols ? g.K : g.M;
  if (bulk) {
    if (!bulk_projection_ok(X, in_dtype, inner, rows, ld)) return false;
  } else if (!make_input_map(&J->map, X, in_dtype, inner, rows, ld)) {
    return false;
  }
  J->src = X;
  J->ld = ld;
  J->inner = inner;
  J->rows = rows;
  J->coef = coef;
  J->out = out;
  J->n_out = cols ? g.N : g.M;
  J->NG = ceil_div(g.K, 8);
  J->pitch = gemm_pitch(g);
  J->Kp_pad = g.Kp_pad;
  J->Kt_pad = g.Kt_pad;
  tma_job_grid(g, cols, &J->units_x, &J->units_y);
  J->nsplit = g.nsplit;
  J->tl = g.tl;
  J->cols = cols;
  if (q) J->q = *q;
  return true;
}

namespace {
using JobsKernel = void (*)(const TmaJob*, const int4*, int64_t, int*);

// The kernel of one (output, tile source, input dtype, l+1); E4M3 output only for
// l+1 in {1, 2, 4, 8} (nullptr otherwise, and nothing instantiated).
template <typename InT, int LP1, bool kQ, bool kBulk>
JobsKernel jobs_kernel_one() {
  if constexpr (kQ && !(LP1 == 1 || LP1 == 2 || LP1 == 4 || LP1 == 8))
    return nullptr;
  else
    return project_tma_jobs_kernel<InT, LP1, kQ, kBulk>;
}

template <bool kQ, bool kBulk, typename InT>
JobsKernel jobs_kernel_lp1(int lp1) {
  switch (lp1) {
    case 1: return jobs_kernel_one<InT, 1, kQ, kBulk>();
    case 2: return jobs_kernel_one<InT, 2, kQ, kBulk>();
    case 3: return jobs_kernel_one<InT, 3, kQ, kBulk>();
    case 4: return jobs_kernel_one<InT, 4, kQ, kBulk>();
    case 5: return jobs_kernel_one<InT, 5, kQ, kBulk>();
    case 6: return jobs_kernel_one<InT, 6, kQ, kBulk>();
    case 7: return jobs_kernel_one<InT, 7, kQ, kBulk>();
    default: return jobs_kernel_one<InT, 8, kQ, kBulk>();
  }
}

template <bool kQ, bool kBulk>
JobsKernel jobs_kernel_for(int in_bf16, int lp1) {
  return in_bf16 ? jobs_kernel_lp1<kQ, kBulk, __nv_bfloat16>(lp1) : jobs_kernel_lp1<kQ, kBulk, float>(lp1);
}
}  // namespace

cudaError_t launch_project_tma_jobs(int in_bf16, int lp1, const TmaJob* jobs, const int4* units, int64_t total,
                                    int* err, int sms, cudaStream_t st, bool quant, bool bulk) {
  if (total == 0) return cudaSuccess;
  if (lp1 < 1 || lp1 > 8) return cudaErrorInvalidValue;
  if (quant && !(lp1 == 1 || lp1 == 2 || lp1 == 4 || lp1 == 8)) return cudaErrorInvalidValue;
  if (bulk && !quant) return cudaErrorInvalidValue;   // bulk tiles feed the E4M3 projections only
  const JobsKernel kern = quant ? (bulk ? jobs_kernel_for<true, true>(in_bf16, lp1) : jobs_kernel_for<true, false>(in_bf16, lp1))
                                : jobs_kernel_for<false, false>(in_bf16, lp1);
  // blocks per SM recorded per device and kernel (0: not yet); a racing repeat is harmless
  static int blocks_per_sm[2][2][2][8][64] = {};
  const int smem = in_bf16 ? (bulk ? PtStages<__nv_bfloat16, true>::kSmem : PtStages<__nv_bfloat16>::kSmem)
                           : (bulk ? PtStages<float, true>::kSmem : PtStages<float>::kSmem);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int& slot = blocks_per_sm[bulk ? 1 : 0][quant ? 1 : 0][in_bf16 ? 1 : 0][lp1 - 1][dev >= 0 && dev < 64 ? dev : 0];
  int nb = dev >= 0 && dev < 64 ? slot : 0;
  if (nb == 0) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kPtThreads, smem);
    if (e != cudaSuccess) return e;
    nb = nb < 1 ? 1 : nb;
    if (dev >= 0 && dev < 64) slot = nb;
  }
  const int64_t slots = static_cast<int64_t>(nb) * sms;
  const int64_t grid = total < slots ? total : slots;
  kern<<<static_cast<unsigned>(grid), kPtThreads, smem, st>>>(jobs, units, total, err);
  return cudaGetLastError();
}

}  // namespace pj
