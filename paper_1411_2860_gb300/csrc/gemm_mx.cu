// Reduced GEMM with FP8 (E4M3) projected components and per-block scales on
// tcgen05 tensor cores (the (l+1) smaller products of Sec. III-B, accumulated
// over blocks as in Eq. 2 and Eq. 8, at the lowest precision of the scaling).
//
// Quantisation (quantize_mx_kernel): every run of 32 consecutive components
// of a row of A_c or B_d (one K block of the block-scaled MMA) gets its own
// power-of-two scale 2^e, e = ceil(log2(amax / 448)), stored as a UE8M0 byte,
// and the components become E4M3(x / 2^e) (round to nearest even, never
// saturating).  With two terms the residual r = x - hi (exact in FP32) is
// quantised the same way with its own scales, and the product keeps
// hi*hi + hi*lo + lo*hi as three K segments, like the BF16 split.
//
// The inputs of the quantiser are the BF16 hi + lo pairs of the projection
// kernels (x to 2^-16 relative), so one projection code path serves both
// precisions.
//
// GEMM (gemm_mx_kernel): tile 128 output columns (rows of B_d, MMA M) x 240
// output rows (rows of A_c, MMA N), 128 components per stage (one 128-byte
// swizzle row of E4M3, four MMAs of K = 32).  Each stage brings its operand
// tiles by TMA and its scale blocks (512 bytes for the 128 B_d rows, 1024 for
// the 240 A_c rows) by bulk copy; the MMA thread moves the scales into TMEM
// with tcgen05.cp (32 x 16-byte rows, repeated in all four lane quadrants)
// right before the four block-scaled MMAs that read them.  Scale blocks are
// laid out per tile and stage as the MMA reads them: row r of a 128-row group
// and K block b at byte (r % 32) * 16 + (r / 32) * 4 + b.
//
// A grouped launch may pick a smaller tile height per instance (a multiple of
// 16), walks a per-CTA tile list, and adds the partial products of tiles that
// cover only part of the K stages to the output (TMA reduction or atomics).
// A single product with an even number of tile columns runs in clusters of two
// CTAs that share each A_c tile (each loads half and multicasts it), as in
// gemm_tc.cu; the scale blocks are loaded by each CTA.
//
// TMEM: accumulators at columns 0 and 256 (240 columns each, so the epilogue
// of one tile overlaps the main loop of the next), scale slots at columns 240
// and 496 (4 columns for the B_d side, 8 for the A_c side), used alternately.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <string.h>

#include "common.hpp"
#include "mx.cuh"
#include "tc.cuh"
#include "tmap.hpp"
#if PJ_CTA_PAIRS
#include "tc_pair.cuh"
#endif

namespace pj {
namespace {

constexpr int XBM = 128;  // output columns per tile (MMA M)
constexpr int XBN = 240;  // output rows per tile (MMA N)
constexpr int XBK = 128;  // components per stage
constexpr int XSTAGES = 4;
constexpr int kXThreads = 192;
constexpr uint32_t kXStageP = XBM * XBK;
constexpr uint32_t kXStageQ = XBN * XBK;
constexpr uint32_t kXStageSF = 512 + 1024;
constexpr int kXEpiRows = 16;
constexpr uint32_t kXStageOut = kXEpiRows * XBM * 4;
constexpr size_t kXSmemBytes = 1024 + XSTAGES * (kXStageP + kXStageQ + kXStageSF) + kXStageOut + 256;
constexpr uint32_t kSlot0 = 240, kSlot1 = 496;
static_assert(kXStageQ % 1024 == 0 && kXStageP % 1024 == 0, "swizzled stages stay 1024-byte aligned");
static_assert(kXSmemBytes <= 232448, "shared memory per block");

struct MxParams {
  MxInst single;
  const MxInst* insts;
  const GemmTile* tiles;    // grouped launch: tiles ordered CTA by CTA
  const int* cta_off;       // grouped launch: tiles of CTA c are [cta_off[c], cta_off[c+1])
  int num_tiles;            // single instance: tiles, walked with a grid stride
  int streamk;              // single instance: CTAs share the K stages of all tiles evenly
  int* err;
};

// The n-th tile of this CTA (instance, coordinates, K-stage range); null past the last.
// kPair (a single instance with an even number of tile columns, clusters of two
// CTAs): the CTAs of a cluster take tile columns 2 c' and 2 c' + 1 of one tile row.
template <bool kPair>
__device__ __forceinline__ const MxInst* mx_tile_of(const MxParams& p, int n, GemmTile& t, int rank) {
  if (kPair && !p.tiles) {
    const int npp = p.single.tiles_n / 2;
    const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
    if (pi >= p.num_tiles / 2) return nullptr;
    t.tj = (pi % npp) * 2 + rank;
    t.ti = pi / npp;
    t.k0 = 0;
    t.k1 = p.single.kc * p.single.nseg;
    t.red = p.single.accum;
    t.pad0 = 0;
    return &p.single;
  }
  if (p.tiles) {
    const int k = p.cta_off[blockIdx.x] + n;
    if (k >= p.cta_off[blockIdx.x + 1]) return nullptr;
    t = p.tiles[k];
    return p.insts + t.inst;
  }
  const int S = p.single.kc * p.single.nseg;
  if (p.streamk) {
    // Stream-K: CTA b owns the K stages [U b / G, U (b+1) / G) of the U = tiles * S
    // stages of the whole product, tile by tile; a tile cut between CTAs adds its
    // partial products into the (zeroed) output.
    const int64_t U = static_cast<int64_t>(p.num_tiles) * S;
    const int64_t u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
    const int64_t start = n == 0 ? u0 : (u0 / S + n) * S;
    if (start >= u1) return nullptr;
    const int tile = static_cast<int>(start / S);
    const int64_t end = u1 < static_cast<int64_t>(tile + 1) * S ? u1 : static_cast<int64_t>(tile + 1) * S;
    t.tj = tile % p.single.tiles_n;
    t.ti = tile / p.single.tiles_n;
    t.k0 = static_cast<int>(start - static_cast<int64_t>(tile) * S);
    t.k1 = static_cast<int>(end - static_cast<int64_t>(tile) * S);
    t.red = (t.k0 != 0 || t.k1 != S || p.single.accum) ? 1 : 0;
    t.pad0 = 0;
    return &p.single;
  }
  const int tile = blockIdx.x + n * gridDim.x;
  if (tile >= p.num_tiles) return nullptr;
  t.tj = tile % p.single.tiles_n;
  t.ti = tile / p.single.tiles_n;
  t.k0 = 0;
  t.k1 = S;
  t.red = p.single.accum;
  t.pad0 = 0;
  return &p.single;
}

// kPair: launched in clusters of two CTAs sharing each Q tile (see mx_tile_of):
// each loads half of the tile's rows and multicasts them to both; every MMA
// commit frees the stage in both CTAs (empty barriers count 2).  Scale blocks
// are loaded by each CTA itself.
template <bool kPair>
__global__ void __launch_bounds__(kXThreads, 1) gemm_mx_kernel(const __grid_constant__ MxParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* sP = sm;
  uint8_t* sQ = sP + XSTAGES * kXStageP;
  uint8_t* sSF = sQ + XSTAGES * kXStageQ;
  uint8_t* stage_out = sSF + XSTAGES * kXStageSF;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage_out + kXStageOut);
  uint64_t* full = bars;
  uint64_t* empty = bars + XSTAGES;
  uint64_t* acc_full = bars + 2 * XSTAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  int* vote = reinterpret_cast<int*>(tslot + 4);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rank = kPair ? static_cast<int>(cluster_ctarank()) : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < XSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kPair ? 2 : 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  if (kPair) cluster_sync_all();  // the peer's barriers exist before any copy or commit reaches them
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: operand tiles by TMA, scale blocks by bulk copy
      int stage = 0;
      uint32_t phase = 0;
      uint32_t last_phase[XSTAGES];
      bool used[XSTAGES];
      for (int s = 0; s < XSTAGES; ++s) used[s] = false;
      bool ok = true;
      GemmTile T{};
      for (int n = 0; ok; ++n) {
        const MxInst* I = mx_tile_of<kPair>(p, n, T, rank);
        if (!I) break;
        const int ti = T.ti, tj = T.tj;
        tma_prefetch(&I->mapP);
        tma_prefetch(&I->mapQ);
        const uint32_t stage_bytes = kXStageP + static_cast<uint32_t>(I->bn) * XBK + kXStageSF;
        for (int kk = T.k0; kk < T.k1; ++kk) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, p.err, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          const int seg = kk / I->kc, kin = kk - seg * I->kc;
          const int xp = I->segP[seg] + kin * XBK, xq = I->segQ[seg] + kin * XBK;
          const uint8_t* sfp = I->sfP + (static_cast<int64_t>(tj) * I->sf_stages + xp / XBK) * 512;
          const uint8_t* sfq = I->sfQ + (static_cast<int64_t>(ti) * I->sf_stages + xq / XBK) * 1024;
          mbar_arrive_expect_tx(&full[stage], stage_bytes);
          tma_load_2d(sP + stage * kXStageP, &I->mapP, &full[stage], xp, tj * XBM);
#if PJ_CTA_PAIRS
          if (kPair) {  // this CTA's half of the Q tile, for both CTAs of the pair
            const int half = I->bn / 2;
            tma_load_2d_mc(sQ + stage * kXStageQ + rank * half * XBK, &I->mapQ, &full[stage], xq,
                           ti * I->bn + rank * half, 0x3);
          } else
#endif
          {
            // (lowered correlation: stage kk of output rows r reads Q rows r + kk)
            if (I->conv_mode)
              tma_load_2d(sQ + stage * kXStageQ, &I->mapQ, &full[stage], 0, ti * I->bn + kk);
            else
              tma_load_2d(sQ + stage * kXStageQ, &I->mapQ, &full[stage], xq, ti * I->bn);
          }
          bulk_load(sSF + stage * kXStageSF, sfp, 512, &full[stage]);
          bulk_load(sSF + stage * kXStageSF + 512, sfq, 1024, &full[stage]);
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == XSTAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      for (int s = 0; s < XSTAGES; ++s)
        if (used[s] && !mbar_wait_drain(&full[s], last_phase[s])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      uint32_t nslot = 0;
      bool ok = true;
      bool issued_any = false;
      GemmTile T{};
      for (int n = 0; ok; ++n, ++it) {
        const MxInst* I = mx_tile_of<kPair>(p, n, T, rank);
        if (!I) break;
        const int acc = it & 1;
        const uint32_t acc_phase = (it >> 1) & 1;
        if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1u, p.err, DEV_TIMEOUT_ACC_FREE)) break;
        tc_fence_after();
        const uint32_t d = tmem + acc * 256;
        for (int kk = T.k0; kk < T.k1; ++kk) {
          if (!mbar_wait(&full[stage], phase, p.err, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t slot = tmem + ((nslot++ & 1u) ? kSlot1 : kSlot0);
          const uint32_t aSF = smem_u32(sSF + stage * kXStageSF);
          tmem_cp_32x128b_warpx4(slot, sdesc_rows16(aSF));
          tmem_cp_32x128b_warpx4(slot + 4, sdesc_rows16(aSF + 512));
          tmem_cp_32x128b_warpx4(slot + 8, sdesc_rows16(aSF + 1024));
          const uint32_t aP = smem_u32(sP + stage * kXStageP);
          const uint32_t aQ = smem_u32(sQ + stage * kXStageQ);
#pragma unroll
          for (int k = 0; k < XBK / 32; ++k)
            umma_mx(d, sdesc_sw128(aP + k * 32, 0), sdesc_sw128(aQ + k * 32, 0), idesc_mx_e4m3(XBM, I->bn, k, k),
                    slot, slot + 4, (kk != T.k0) || (k != 0));
          issued_any = true;
#if PJ_CTA_PAIRS
          if (kPair)
            umma_commit_mc(&empty[stage], 0x3);
          else
#endif
            umma_commit(&empty[stage]);
          if (++stage == XSTAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) umma_commit(&acc_full[acc]);
      }
      if (issued_any) {
        umma_commit(drain);
        if (!mbar_wait_drain(drain, 0)) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> registers -> shared staging -> TMA store
    const int q = warp & 3;
    const bool leader = warp == 2 && lane == 0;
    bool pending = false;
    int it = 0;
    GemmTile T{};
    for (int n = 0;; ++n, ++it) {
      const MxInst* I = mx_tile_of<kPair>(p, n, T, rank);
      if (!I) break;
      const int ti = T.ti, tj = T.tj;
      const bool red = T.red != 0;
      const int acc = it & 1;
      const uint32_t acc_phase = (it >> 1) & 1;
      const bool okw = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], acc_phase, p.err, DEV_TIMEOUT_ACC));
      if (lane == 0) vote[(it & 1) * 4 + q] = okw ? 1 : 0;
      named_barrier(1, 128);
      const int* v = vote + (it & 1) * 4;
      if (!(v[0] && v[1] && v[2] && v[3])) break;
      tc_fence_after();
      const int M = I->M, N = I->N;
      const int jl = q * 32 + lane;
      const int j = tj * XBM + jl;
      const bool jok = j < N;
      for (int c0 = 0; c0 < I->bn; c0 += kXEpiRows) {
        uint32_t r[kXEpiRows];
        tmem_ld_x16(tmem + acc * 256 + c0 + (static_cast<uint32_t>(q * 32) << 16), r);
        tmem_wait_ld();
        const int i0 = ti * I->bn + c0;
        if (i0 >= M) continue;
        if (I->conv_mode) {
          // lowered correlation: element (i, j) is output sample i * 128 + j of this phase
          float* Y = static_cast<float*>(I->Y);
#pragma unroll
          for (int u = 0; u < kXEpiRows; ++u) {
            const int64_t flat = static_cast<int64_t>(i0 + u) * XBM + j;
            if (jok && flat < I->conv_limit) __stcs(Y + flat * I->conv_stride, __uint_as_float(r[u]));
          }
        } else if (I->tma_out && (tj + 1) * XBM <= I->tma_cols) {
          if (leader && pending) bulk_wait_read_all();
          named_barrier(1, 128);
          if (I->out_bf16) {
            __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(stage_out);
#pragma unroll
            for (int u = 0; u < kXEpiRows; ++u) st[u * XBM + jl] = __float2bfloat16_rn(__uint_as_float(r[u]));
          } else {
            float* st = reinterpret_cast<float*>(stage_out);
#pragma unroll
            for (int u = 0; u < kXEpiRows; ++u) st[u * XBM + jl] = __uint_as_float(r[u]);
          }
          fence_proxy_async_smem();
          named_barrier(1, 128);
          if (leader) {
            if (red)
              tma_reduce_add_2d(&I->mapY, stage_out, tj * XBM, i0);
            else
              tma_store_2d(&I->mapY, stage_out, tj * XBM, i0);
            bulk_commit_group();
            pending = true;
          }
        } else if (I->out_bf16) {
          __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(I->Y);
#pragma unroll
          for (int u = 0; u < kXEpiRows; ++u)
            if (jok && i0 + u < M)
              Y[static_cast<int64_t>(i0 + u) * I->ldy + j] = __float2bfloat16_rn(__uint_as_float(r[u]));
        } else if (red) {
          float* Y = static_cast<float*>(I->Y);
#pragma unroll
          for (int u = 0; u < kXEpiRows; ++u)
            if (jok && i0 + u < M) atomicAdd(Y + static_cast<int64_t>(i0 + u) * I->ldy + j, __uint_as_float(r[u]));
        } else {
          float* Y = static_cast<float*>(I->Y);
#pragma unroll
          for (int u = 0; u < kXEpiRows; ++u)
            if (jok && i0 + u < M) __stcs(Y + static_cast<int64_t>(i0 + u) * I->ldy + j, __uint_as_float(r[u]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
    }
    if (leader && pending) bulk_wait_all();
  }

  tc_fence_before();
  __syncthreads();
  // Neither CTA of a pair leaves while the other's MMAs may still arrive on its barriers.
  if (kPair) cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------ quantiser --

// Quantises x[0..31] with scale 2^e into 32 E4M3 bytes (q) and returns the
// dequantised values in x (x becomes the residual x - deq when `residual`).
__device__ __forceinline__ void quant32(float (&x)[32], int e, uint32_t (&q)[8], bool residual) {
  const float inv = ldexpf(1.0f, -e), s = ldexpf(1.0f, e);
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const uint32_t a = e4m3x2(x[4 * w], x[4 * w + 1], inv);
    const uint32_t b = e4m3x2(x[4 * w + 2], x[4 * w + 3], inv);
    q[w] = a | (b << 16);
    if (residual) {
      const float2 da = e4m3x2_value(a);
      const float2 db = e4m3x2_value(b);
      x[4 * w] -= da.x * s;
      x[4 * w + 1] -= da.y * s;
      x[4 * w + 2] -= db.x * s;
      x[4 * w + 3] -= db.y * s;
    }
  }
}

// Quantises unit u of one side: row u / (Kq_pad / 32), run u mod (Kq_pad / 32).
__device__ __forceinline__ void quantize_unit(const MxQuantSide& a, int64_t u) {
  const int qsplit = a.qsplit;
  const int64_t nch = a.Kq_pad / 32;
  const int64_t r = u / nch, c = u - r * nch;
  const int64_t lo_chunk = a.Kq_pad / 32;
  if (r >= a.rows) {  // padding rows of the last tile: unit scales, no data
    a.sf[mx_sf_offset(a, r, c)] = 127;
    if (qsplit > 1) a.sf[mx_sf_offset(a, r, lo_chunk + c)] = 127;
    return;
  }
  float x[32];
  if (c * 32 < a.Kp_pad) {
    const uint4* hp = reinterpret_cast<const uint4*>(a.src + r * a.src_pitch + c * 32);
    const uint4* lp = reinterpret_cast<const uint4*>(a.src + r * a.src_pitch + a.Kp_pad + c * 32);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint4 h = hp[v], l = lp[v];
      const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        x[8 * v + 2 * w] = __uint_as_float(hw[w] << 16) + __uint_as_float(lw[w] << 16);
        x[8 * v + 2 * w + 1] = __uint_as_float(hw[w] & 0xffff0000u) + __uint_as_float(lw[w] & 0xffff0000u);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = 0.0f;
  }
  float amax = 0.0f;
#pragma unroll
  for (int k = 0; k < 32; ++k) amax = fmaxf(amax, fabsf(x[k]));
  const int e = mx_exponent(amax);
  uint32_t q[8];
  quant32(x, e, q, qsplit > 1);
  uint8_t* row = a.dst + r * a.dst_pitch;
  uint4* o = reinterpret_cast<uint4*>(row + c * 32);
  o[0] = make_uint4(q[0], q[1], q[2], q[3]);
  o[1] = make_uint4(q[4], q[5], q[6], q[7]);
  a.sf[mx_sf_offset(a, r, c)] = static_cast<uint8_t>(e + 127);
  if (qsplit > 1) {
    float amax2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) amax2 = fmaxf(amax2, fabsf(x[k]));
    const int e2 = mx_exponent(amax2);
    quant32(x, e2, q, false);
    uint4* o2 = reinterpret_cast<uint4*>(row + a.Kq_pad + c * 32);
    o2[0] = make_uint4(q[0], q[1], q[2], q[3]);
    o2[1] = make_uint4(q[4], q[5], q[6], q[7]);
    a.sf[mx_sf_offset(a, r, lo_chunk + c)] = static_cast<uint8_t>(e2 + 127);
  }
}

__global__ void __launch_bounds__(256) quantize_mx_kernel(const MxQuantSide s0, const MxQuantSide s1, int64_t n0,
                                                          int64_t total) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= total) return;
  if (t < n0)
    quantize_unit(s0, t);
  else
    quantize_unit(s1, t - n0);
}

// Batched form: block b belongs to side job_of[b], whose units start at block block0.
__global__ void __launch_bounds__(256) quantize_mx_jobs_kernel(const MxQuantSide* __restrict__ sides,
                                                               const int* __restrict__ job_of) {
  const MxQuantSide& a = sides[job_of[blockIdx.x]];
  const int64_t u = (static_cast<int64_t>(blockIdx.x) - a.block0) * blockDim.x + threadIdx.x;
  if (u < a.tiles * a.tile_rows * (a.Kq_pad / 32)) quantize_unit(a, u);
}

cudaError_t set_mx_smem_attr() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(gemm_mx_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kXSmemBytes));
#if PJ_CTA_PAIRS
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_mx_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kXSmemBytes));
#endif
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

}  // namespace

size_t mx_sf_bytes(int64_t rows, int side_q, int64_t Kq_pad, int qsplit, int bn) {
  const int64_t nst = Kq_pad * qsplit / XBK;
  return static_cast<size_t>(ceil_div(rows, side_q ? bn : XBM) * nst * (side_q ? 1024 : 512));
}

MxQuantSide make_mx_side(const uint16_t* src, int64_t Kp_pad, int64_t rows, uint8_t* dst, int64_t Kq_pad, int qsplit,
                         uint8_t* sf, int side_q, int bn) {
  MxQuantSide a;
  a.src = src;
  a.src_pitch = 2 * Kp_pad;
  a.Kp_pad = Kp_pad;
  a.rows = rows;
  a.dst = dst;
  a.dst_pitch = Kq_pad * qsplit;
  a.Kq_pad = Kq_pad;
  a.sf = sf;
  a.tile_rows = side_q ? bn : XBM;
  a.atoms = side_q ? 2 : 1;
  a.sf_stages = Kq_pad * qsplit / XBK;
  a.tiles = ceil_div(rows, a.tile_rows);
  a.qsplit = qsplit;
  a.block0 = 0;
  return a;
}

int64_t mx_side_blocks(const MxQuantSide& a) { return ceil_div(a.tiles * a.tile_rows * (a.Kq_pad / 32), 256); }

cudaError_t launch_quantize_mx_jobs(const MxQuantSide* sides, const int* job_of, int64_t blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  quantize_mx_jobs_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(sides, job_of);
  return cudaGetLastError();
}

cudaError_t launch_quantize_mx(const MxQuantSide* a, const MxQuantSide* b, cudaStream_t st) {
  MxQuantSide none{};
  const MxQuantSide& s0 = a ? *a : (b ? *b : none);
  const MxQuantSide& s1 = (a && b) ? *b : none;
  const int64_t n0 = (a || b) ? s0.tiles * s0.tile_rows * (s0.Kq_pad / 32) : 0;
  const int64_t n1 = (a && b) ? s1.tiles * s1.tile_rows * (s1.Kq_pad / 32) : 0;
  const int64_t total = n0 + n1;
  if (total == 0) return cudaSuccess;
  quantize_mx_kernel<<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(s0, s1, n0, total);
  return cudaGetLastError();
}

bool build_mx_inst(const MxGemmArgs& a, MxInst* I) {
  memset(I, 0, sizeof(MxInst));
  {
    const uint64_t dims[2] = {static_cast<uint64_t>(a.pitch), static_cast<uint64_t>(a.rowsP)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.pitch)};
    const uint32_t box[2] = {XBK, XBM};
    if (!make_tmap_u8_sw128(&I->mapP, a.P, 2, dims, strides, box)) return false;
  }
  {
    // (a lowered correlation's Q: its q_rows rows of 128 components)
    const int64_t qp = a.conv_mode ? a.q_pitch : a.pitch, qr = a.conv_mode ? a.q_rows : a.rowsQ;
    const uint64_t dims[2] = {static_cast<uint64_t>(qp), static_cast<uint64_t>(qr)};
    const uint64_t strides[1] = {static_cast<uint64_t>(qp)};
    const uint32_t box[2] = {XBK, static_cast<uint32_t>(a.pair ? a.bn / 2 : a.bn)};
    if (!make_tmap_u8_sw128(&I->mapQ, a.Q, 2, dims, strides, box)) return false;
  }
  I->conv_mode = a.conv_mode;
  I->conv_stride = a.conv_stride;
  I->conv_limit = a.conv_limit;
  I->bn = a.bn;
  I->accum = (a.accum && a.out_dtype != PJ_BF16) ? 1 : 0;
  I->sfP = a.sfP;
  I->sfQ = a.sfQ;
  I->sf_stages = a.pitch / XBK;
  I->Y = a.Y;
  I->ldy = a.ldy;
  I->out_bf16 = a.out_dtype == PJ_BF16;
  I->M = static_cast<int>(a.rowsQ);
  I->N = static_cast<int>(a.rowsP);
  I->kc = static_cast<int>(a.Kq_pad / XBK);
  I->nseg = a.qsplit == 1 ? 1 : 3;
  // hi*hi + hi(B_d)*lo(A_c) + lo(B_d)*hi(A_c)
  I->segP[0] = 0; I->segQ[0] = 0;
  I->segP[1] = 0; I->segQ[1] = static_cast<int>(a.Kq_pad);
  I->segP[2] = static_cast<int>(a.Kq_pad); I->segQ[2] = 0;
  I->tiles_n = static_cast<int>(ceil_div(a.rowsP, XBM));
  I->tiles_m = static_cast<int>(ceil_div(a.rowsQ, a.bn));
  const size_t es = I->out_bf16 ? 2 : 4;
  I->tma_out = 0;
  // a TMA store writes the whole 16-byte chunk of a row's last element: a ragged
  // last tile column of a row that does not end on 16 bytes is stored element-wise
  I->tma_cols = (a.rowsP * static_cast<int64_t>(es)) % 16 ? static_cast<int>(a.rowsP) : (1 << 30);
  if ((a.ldy * es) % 16 == 0 && reinterpret_cast<uintptr_t>(a.Y) % 16 == 0) {
    const uint64_t dims[2] = {static_cast<uint64_t>(a.rowsP), static_cast<uint64_t>(a.rowsQ)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.ldy) * es};
    const uint32_t box[2] = {XBM, kXEpiRows};
    I->tma_out = (I->out_bf16 ? make_tmap_bf16_plain(&I->mapY, a.Y, 2, dims, strides, box)
                              : make_tmap_f32(&I->mapY, a.Y, 2, dims, strides, box)) ? 1 : 0;
  }
  return true;
}

cudaError_t launch_gemm_mx(const MxGemmArgs& a_in, int* err, int num_sms, cudaStream_t st) {
  if (a_in.rowsQ == 0 || a_in.rowsP == 0) return cudaSuccess;
  // The tile height is fixed by the scale-block layout the quantiser wrote (a.bn).
  MxGemmArgs a = a_in;
  const int64_t tiles_n = ceil_div(a.rowsP, XBM), tiles = tiles_n * ceil_div(a.rowsQ, a.bn);
  const int stages = static_cast<int>(a.Kq_pad / XBK) * (a.qsplit == 1 ? 1 : 3);
  const bool streamk = a.out_dtype != PJ_BF16 && use_stream_k(static_cast<int>(tiles), stages, num_sms);
  // CTA pairs share the Q tiles when the tile columns pair up (half-tiles of whole 8-row atoms).
  a.pair = PJ_CTA_PAIRS && !streamk && tiles_n % 2 == 0 && a.bn % 16 == 0 && num_sms >= 2;
  MxParams p;
  if (!build_mx_inst(a, &p.single)) return cudaErrorInvalidValue;
  p.insts = nullptr;
  p.tiles = nullptr;
  p.cta_off = nullptr;
  p.num_tiles = p.single.tiles_n * p.single.tiles_m;
  p.err = err;
  cudaError_t e = set_mx_smem_attr();
  if (e != cudaSuccess) return e;
  int grid = p.num_tiles < num_sms ? p.num_tiles : num_sms;
  p.streamk = 0;
  if (streamk) {
    // partial tiles add into the output: cleared first unless the product is itself added
    if (!a.accum) e = cudaMemset2DAsync(a.Y, a.ldy * 4, 0, a.rowsP * 4, a.rowsQ, st);
    if (e != cudaSuccess) return e;
    p.streamk = 1;
    grid = num_sms;
  }
#if PJ_CTA_PAIRS
  if (a.pair) {
    const int pairs = p.num_tiles / 2, slots = num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(2 * (pairs < slots ? pairs : slots)));
    cfg.blockDim = dim3(kXThreads);
    cfg.dynamicSmemBytes = kXSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gemm_mx_kernel<true>, p);
  }
#endif
  gemm_mx_kernel<false><<<grid, kXThreads, kXSmemBytes, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gemm_mx_grouped(const MxInst* insts, const GemmTile* tiles, const int* cta_off, int ctas,
                                   int* err, cudaStream_t st) {
  if (ctas == 0) return cudaSuccess;
  MxParams p;
  memset(&p.single, 0, sizeof(MxInst));
  p.insts = insts;
  p.tiles = tiles;
  p.cta_off = cta_off;
  p.num_tiles = 0;
  p.streamk = 0;
  p.err = err;
  cudaError_t e = set_mx_smem_attr();
  if (e != cudaSuccess) return e;
  gemm_mx_kernel<false><<<ctas, kXThreads, kXSmemBytes, st>>>(p);
  return cudaGetLastError();
}

}  // namespace pj
