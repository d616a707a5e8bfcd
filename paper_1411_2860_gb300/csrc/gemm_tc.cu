// Reduced GEMM on tcgen05 tensor cores (the (l+1) smaller products of
// Sec. III-B, Fig. 5, accumulated over blocks as in Eq. 2 and Eq. 8).
//
// Y[i][j] = sum_k A_c[i][k] B_d[j][k] over the reduced inner dimension k
// (all blocks and kept projections; with split components, three passes
// hi*hi + hi*lo + lo*hi).  The per-block partial products are summed in the
// FP32 TMEM accumulator as part of the MMA K loop.
//
// Tile: 128 output columns (rows of B_d, the MMA M side) x up to 256 output
// rows (rows of A_c, the MMA N side; a grouped launch picks the height per
// instance, a multiple of 32), K step 64 (one 128-byte swizzle row).
// Persistent CTAs, one per SM; warp 0 issues TMA loads, warp 1 issues UMMA,
// warps 2-5 drain the two TMEM accumulators (2 x 256 columns) so the epilogue
// of one tile overlaps the main loop of the next.  TMEM lane = output column,
// so each warp's stores of one output row are 128 contiguous bytes.
//
// A tile moves (128 + rows) x 128 bytes from L2 per K stage; at the tensor
// rate that is more than the SMs can draw from L2, so K-major products run in
// clusters of two CTAs on neighbouring tile columns of one tile row: each CTA
// loads half of the shared A_c rows and multicasts them to both (kPair).
// With the hi/lo split, the three segments are walked stage by stage, so the
// hi tiles of a K chunk are read again while they are still in L2.
//
// A grouped launch walks a per-CTA tile list planned on the host; a tile may
// cover only a range of the K stages of its instance (a split reduced
// dimension), in which case its partial product is added to the output by a
// TMA reduction (or FP32 atomics) instead of stored.
#include <cuda_bf16.h>
#include <string.h>

#include "common.hpp"
#include "gemm_epi.cuh"
#include "tc.cuh"
#include "tmap.hpp"
#if PJ_CTA_PAIRS
#include "tc_pair.cuh"
#endif

namespace pj {
namespace {

constexpr int BM = 128;  // output columns per tile (MMA M)
constexpr int BN = 256;  // output rows per tile (MMA N)
constexpr int BK = 64;
constexpr int STAGES = 4;
constexpr int kThreads = 192;
constexpr uint32_t kStageP = BM * BK * 2;
constexpr uint32_t kStageQ = BN * BK * 2;
constexpr uint32_t kStageOut = 32 * BM * 4;          // output staging: 32 rows x 128 columns (FP32 max)
constexpr size_t kSmemBytes = 1024 + STAGES * (kStageP + kStageQ) + kStageOut + 256;

struct GemmParams {
  GemmInst single;           // the instance when `tiles` is null
  const GemmInst* insts;     // grouped launch: instance table in global memory
  const GemmTile* tiles;     // grouped launch: tiles ordered CTA by CTA (null for a single instance)
  const int* cta_off;        // grouped launch: tiles of CTA c are [cta_off[c], cta_off[c+1])
  int num_tiles;             // single instance: tiles, walked with a grid stride
  int streamk;               // single instance: CTAs share the K stages of all tiles evenly
  int stall;                 // failure-detection self-test: the producer stops after this many stages (-1: never)
  int* err;
  ExpandArgs ex;             // single instance: expansion to samples in the epilogue (mode 0: none)
};

// The n-th tile of this CTA: instance, coordinates and K-stage range; false past the last.
// kPair (a single instance with an even number of tile columns, clusters of two CTAs):
// the CTAs of cluster c take the tile columns 2 c' and 2 c' + 1 (by cluster rank) of the
// same tile row, so both read the same rows of A_c.
template <bool kPair>
__device__ __forceinline__ const GemmInst* tile_of(const GemmParams& p, int n, GemmTile& t, int rank) {
  if (kPair && !p.tiles) {
    const int npp = p.single.tiles_n / 2;
    const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
    if (pi >= p.num_tiles / 2) return nullptr;
    t.tj = (pi % npp) * 2 + rank;
    t.ti = pi / npp;
    t.k0 = 0;
    t.k1 = p.single.kc;
    t.red = 0;
    t.pad0 = 0;
    return &p.single;
  }
  if (p.tiles) {
    const int k = p.cta_off[blockIdx.x] + n;
    if (k >= p.cta_off[blockIdx.x + 1]) return nullptr;
    t = p.tiles[k];
    return p.insts + t.inst;
  }
  const int S = p.single.kc;
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
    t.red = (t.k0 != 0 || t.k1 != S) ? 1 : 0;
    t.pad0 = 0;
    return &p.single;
  }
  const int tile = blockIdx.x + n * gridDim.x;
  if (tile >= p.num_tiles) return nullptr;
  t.tj = tile % p.single.tiles_n;
  t.ti = tile / p.single.tiles_n;
  t.k0 = 0;
  t.k1 = S;
  t.red = 0;
  t.pad0 = 0;  // no pair flags: the epilogue's stores (and its barriers) run in every warp
  return &p.single;
}

// kMN: the launch may hold MN-major operands (the K-major instantiation carries
// none of their branches).  kPair: launched in clusters of two CTAs that share
// every Q tile (see tile_of): each CTA loads half of the tile's rows and the
// copy is multicast to both, so the pair reads the rows of A_c once.  A stage
// is then free only when both CTAs' MMAs have read it: every MMA commit
// arrives on the stage's empty barrier in both CTAs (initial count 2).
template <bool kMN, bool kPair>
__global__ void __launch_bounds__(kThreads, 1) gemm_tc_kernel(const __grid_constant__ GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* sP = sm;
  uint8_t* sQ = sm + STAGES * kStageP;
  uint8_t* stage = sQ + STAGES * kStageQ;              // output staging
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + kStageOut);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* acc_full = bars + 2 * STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  int* vote = reinterpret_cast<int*>(tslot + 4);       // [2][4] epilogue warps' wait outcomes

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rank = kPair ? static_cast<int>(cluster_ctarank()) : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
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
      // ---------------- TMA producer
      int stage = 0;
      uint32_t phase = 0;
      uint32_t last_phase[STAGES];
      bool used[STAGES];
      for (int s = 0; s < STAGES; ++s) used[s] = false;
      bool ok = true;
      int issued = 0;
      GemmTile T{};
      for (int n = 0; ok; ++n) {
        const GemmInst* I = tile_of<kPair>(p, n, T, rank);
        if (!I) break;
        const int ti = T.ti, tj = T.tj;
        tma_prefetch(&I->mapP);
        tma_prefetch(&I->mapQ);
        const uint32_t stage_bytes = kStageP + static_cast<uint32_t>(I->bn) * BK * 2;
        const int qchunks = I->bn / 64;
        for (int kk = T.k0; kk < T.k1; ++kk, ++issued) {
          if (issued == p.stall) {  // self-test only: the consumers' bounded waits must run out
            ok = false;
            break;
          }
          if (!mbar_wait(&empty[stage], phase ^ 1u, p.err, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          int seg = 0, kin = kk;
          if (I->ilv) {  // three equal segments taken stage by stage: a K chunk's hi tiles are reused at once
            seg = kk % 3;
            kin = kk / 3;
          } else {
            while (seg + 1 < I->nseg && kin >= I->segKc[seg]) kin -= I->segKc[seg++];
          }
          // Row-split mode: Q row r, K chunk k lives at row r + k/2, column 64 (k mod 2) of
          // a 128-wide view (the signal segments of a lowered correlation); there a
          // segment's Q offset counts rows (the split residual rows follow the hi rows).
          const int qx = I->conv_mode ? (kin & 1) * BK : I->segQ[seg] + kin * BK;
          const int qy = I->conv_mode ? ti * I->bn + (kin >> 1) + I->segQ[seg] : ti * I->bn;
          mbar_arrive_expect_tx(&full[stage], stage_bytes);
          if (kMN && I->mnP) {  // 64-wide MN chunks of 64 K rows (8 KB each)
            tma_load_2d(sP + stage * kStageP, &I->mapP, &full[stage], tj * BM, I->segP[seg] + kin * BK);
            tma_load_2d(sP + stage * kStageP + 8192, &I->mapP, &full[stage], tj * BM + 64, I->segP[seg] + kin * BK);
          } else {
            tma_load_2d(sP + stage * kStageP, &I->mapP, &full[stage], I->segP[seg] + kin * BK, tj * BM);
          }
          if (kMN && I->mnQ) {
#if PJ_CTA_PAIRS
            if (kPair) {  // this CTA's half of the Q chunks, for both CTAs of the pair
              const int hc = qchunks / 2;
              for (int c = rank * hc; c < (rank + 1) * hc; ++c)
                tma_load_2d_mc(sQ + stage * kStageQ + c * 8192, &I->mapQ, &full[stage], ti * I->bn + 64 * c,
                               I->segQ[seg] + kin * BK, 0x3);
            } else
#endif
            for (int c = 0; c < qchunks; ++c)
              tma_load_2d(sQ + stage * kStageQ + c * 8192, &I->mapQ, &full[stage], ti * I->bn + 64 * c,
                          I->segQ[seg] + kin * BK);
#if PJ_CTA_PAIRS
          } else if (kPair && !(T.pad0 & 1)) {
            // this CTA's half of the Q tile, for both CTAs of the pair
            const int half = I->bn / 2;
            tma_load_2d_mc(sQ + stage * kStageQ + rank * half * (BK * 2), &I->mapQ, &full[stage], qx,
                           qy + rank * half, 0x3);
#endif
          } else if (kPair) {
            // a tile of its own (grouped launch): both halves for this CTA only
            const int half = I->bn / 2;
            tma_load_2d(sQ + stage * kStageQ, &I->mapQ, &full[stage], qx, qy);
            tma_load_2d(sQ + stage * kStageQ + half * (BK * 2), &I->mapQ, &full[stage], qx, qy + half);
          } else {
            tma_load_2d(sQ + stage * kStageQ, &I->mapQ, &full[stage], qx, qy);
          }
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // Every issued copy must land before the CTA may exit.
      for (int s = 0; s < STAGES; ++s)
        if (used[s] && !mbar_wait_drain(&full[s], last_phase[s])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- UMMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      bool ok = true;
      bool issued_any = false;
      GemmTile T{};
      for (int n = 0; ok; ++n, ++it) {
        const GemmInst* I = tile_of<kPair>(p, n, T, rank);
        if (!I) break;
        const bool mnP = kMN && I->mnP != 0, mnQ = kMN && I->mnQ != 0;
        const uint32_t idesc = idesc_bf16_f32(BM, I->bn) | (static_cast<uint32_t>(mnP) << 15) |
                               (static_cast<uint32_t>(mnQ) << 16);
        const int acc = it & 1;
        const uint32_t acc_phase = (it >> 1) & 1;
        if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1u, p.err, DEV_TIMEOUT_ACC_FREE)) break;
        tc_fence_after();
        const uint32_t d = tmem + acc * BN;
        for (int kk = T.k0; kk < T.k1; ++kk) {
          if (!mbar_wait(&full[stage], phase, p.err, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aP = smem_u32(sP + stage * kStageP);
          const uint32_t aQ = smem_u32(sQ + stage * kStageQ);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t dp = mnP ? sdesc_sw128_mn(aP + k * 2048, 8192) : sdesc_sw128(aP + k * 32, 0);
            const uint64_t dq = mnQ ? sdesc_sw128_mn(aQ + k * 2048, 8192) : sdesc_sw128(aQ + k * 32, 0);
            umma_f16(d, dp, dq, idesc, (kk != T.k0) || (k != 0));
          }
          issued_any = true;
#if PJ_CTA_PAIRS
          if (kPair)
            umma_commit_mc(&empty[stage], 0x3);
          else
#endif
            umma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) umma_commit(&acc_full[acc]);
      }
      // Commit only behind issued MMAs: a commit with nothing to track is never issued.
      if (issued_any) {
        umma_commit(drain);
        if (!mbar_wait_drain(drain, 0)) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> registers -> shared staging -> TMA store
    // (direct stores when Y's pitch does not allow TMA; or the expansion to
    // samples of a gradient product, written straight from registers)
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const bool leader = warp == 2 && lane == 0;
    bool pending = false;
    __shared__ float s_coef[64];
    // read once: the stores go through generic pointers, after which values read
    // through a pointer to the parameters would be read again
    const ExpandArgs ex = p.ex;
    if (ex.mode) {
      const int ncoef = 8 * ex.lp1;
      for (int e = threadIdx.x - 64; e < ncoef; e += 128) s_coef[e] = ex.coef[e];
      named_barrier(1, 128);
    }
    int it = 0;
    GemmTile T{};
    for (int n = 0;; ++n, ++it) {
      const GemmInst* I = tile_of<kPair>(p, n, T, rank);
      if (!I) break;
      const int ti = T.ti, tj = T.tj;
      const bool red = T.red != 0;
      const int acc = it & 1;
      const uint32_t acc_phase = (it >> 1) & 1;
      const bool okw = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], acc_phase, p.err, DEV_TIMEOUT_ACC));
      // The four epilogue warps take the same decision, so none is left alone at a barrier.
      if (lane == 0) vote[(it & 1) * 4 + q] = okw ? 1 : 0;
      named_barrier(1, 128);
      const int* v = vote + (it & 1) * 4;
      if (!(v[0] && v[1] && v[2] && v[3])) break;
      tc_fence_after();
      const int M = I->M, N = I->N;
      const int jl = q * 32 + lane;
      const int j = tj * BM + jl;
      const bool jok = j < N;
      if (ex.mode) {
        // Y[i][j] (i: row of Q, j: row of P) expanded to samples: mode 1 has the
        // components on j (N = their count), mode 2 on i (M = their count).
        const int ncomp = ex.mode == 1 ? N : M;
        expand_tile(tmem + acc * BN + (static_cast<uint32_t>(q * 32) << 16), I->bn, ex, s_coef, lane, j, ncomp,
                    ti * I->bn, M, j, jok);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[acc]);
        continue;
      }
      // a stand-in tile of a pair (grouped launch) writes nothing
      for (int c0 = 0; c0 < ((T.pad0 & 2) ? 0 : I->bn); c0 += 32) {
        uint32_t r[32];
        tmem_ld_x32(tmem + acc * BN + c0 + (static_cast<uint32_t>(q * 32) << 16), r);
        tmem_wait_ld();
        const int i0 = ti * I->bn + c0;
        if (i0 >= M) continue;  // uniform: no rows of this chunk exist
        if (I->tma_out && i0 + 32 <= I->tma_rows && (tj + 1) * BM <= I->tma_cols) {
          if (leader && pending) bulk_wait_read_all();
          named_barrier(1, 128);  // staging free
          if (I->out_bf16) {
            __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(stage);
#pragma unroll
            for (int u = 0; u < 32; ++u) st[u * BM + jl] = __float2bfloat16_rn(__uint_as_float(r[u]));
          } else {
            float* st = reinterpret_cast<float*>(stage);
#pragma unroll
            for (int u = 0; u < 32; ++u) st[u * BM + jl] = __uint_as_float(r[u]);
          }
          fence_proxy_async_smem();
          named_barrier(1, 128);  // staging written
          if (leader) {
            if (red)
              tma_reduce_add_2d(&I->mapY, stage, tj * BM, i0);
            else
              tma_store_2d(&I->mapY, stage, tj * BM, i0);
            bulk_commit_group();
            pending = true;
          }
        } else if (I->conv_mode) {
          // lowered correlation: element (i, j) is output sample i * 128 + j of this phase
          float* Y = static_cast<float*>(I->Y);
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int64_t flat = static_cast<int64_t>(i0 + u) * BM + j;
            if (jok && flat < I->conv_limit) __stcs(Y + flat * I->conv_stride, __uint_as_float(r[u]));
          }
        } else if (I->out_bf16) {
          __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(I->Y);
          const int64_t ldy = I->ldy;
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < M) Y[static_cast<int64_t>(i0 + u) * ldy + j] = __float2bfloat16_rn(__uint_as_float(r[u]));
        } else if (red) {
          float* Y = static_cast<float*>(I->Y);
          const int64_t ldy = I->ldy;
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < M) atomicAdd(Y + static_cast<int64_t>(i0 + u) * ldy + j, __uint_as_float(r[u]));
        } else {
          float* Y = static_cast<float*>(I->Y);
          const int64_t ldy = I->ldy;
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < M) __stcs(Y + static_cast<int64_t>(i0 + u) * ldy + j, __uint_as_float(r[u]));
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

}  // namespace

bool build_gemm_inst(const GemmTcArgs& a, GemmInst* I) {
  memset(I, 0, sizeof(GemmInst));
  if ((a.mnQ && (a.bn % 64 || a.conv_mode)) || (a.mnP && a.conv_mode)) return false;
  if (a.mnP) {  // stored as xdim K rows of rowsP values: boxes of 64 values x 64 K rows
    const uint64_t dims[2] = {static_cast<uint64_t>(a.rowsP), static_cast<uint64_t>(a.xdim)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.ldp) * 2};
    const uint32_t box[2] = {64, BK};
    if (!make_tmap_bf16(&I->mapP, a.P, 2, dims, strides, box)) return false;
  } else {
    const uint64_t dims[2] = {static_cast<uint64_t>(a.xdim), static_cast<uint64_t>(a.rowsP)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.ldp) * 2};
    const uint32_t box[2] = {BK, BM};
    if (!make_tmap_bf16(&I->mapP, a.P, 2, dims, strides, box)) return false;
  }
  if (a.mnQ) {
    const uint64_t dims[2] = {static_cast<uint64_t>(a.rowsQ), static_cast<uint64_t>(a.xdim)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.ldq) * 2};
    const uint32_t box[2] = {64, BK};
    if (!make_tmap_bf16(&I->mapQ, a.Q, 2, dims, strides, box)) return false;
  } else {
    const uint64_t dims[2] = {static_cast<uint64_t>(a.conv_mode ? 128 : a.xdim),
                              static_cast<uint64_t>(a.conv_mode ? a.q_rows_alloc : a.rowsQ)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.ldq) * 2};
    const uint32_t box[2] = {BK, static_cast<uint32_t>(a.pair ? a.bn / 2 : a.bn)};
    if (!make_tmap_bf16(&I->mapQ, a.Q, 2, dims, strides, box)) return false;
  }
  I->bn = a.bn;
  I->mnQ = a.mnQ;
  I->mnP = a.mnP;
  I->Y = a.Y;
  I->ldy = a.ldy;
  I->out_bf16 = a.out_dtype == PJ_BF16;
  I->M = static_cast<int>(a.rowsQ);
  I->N = static_cast<int>(a.rowsP);
  I->nseg = a.nseg;
  I->kc = 0;
  for (int s = 0; s < 3; ++s) {
    I->segP[s] = static_cast<int>(a.segP[s]);
    I->segQ[s] = static_cast<int>(a.segQ[s]);
    I->segKc[s] = s < a.nseg ? static_cast<int>(ceil_div(a.segK[s] ? a.segK[s] : a.kdim, BK)) : 0;
    I->kc += I->segKc[s];
  }
  // The plain split's three segments (hi*hi, hi*lo, lo*hi) share their hi tiles:
  // interleaved, each K chunk's hi tiles are read again while still in L2.
  I->ilv = (a.nseg == 3 && !a.conv_mode && I->segKc[0] == I->segKc[1] && I->segKc[1] == I->segKc[2]) ? 1 : 0;
  I->tiles_n = static_cast<int>(ceil_div(a.rowsP, BM));
  I->conv_mode = a.conv_mode;
  I->conv_stride = a.conv_stride;
  I->conv_limit = a.conv_limit;
  I->tma_out = 0;
  I->tma_rows = static_cast<int>(a.rowsQ);
  I->tma_cols = 1 << 30;
  const size_t es = I->out_bf16 ? 2 : 4;
  if (a.conv_mode) {
    // contiguous output rows of 128 samples only when samples are adjacent in memory
    const int64_t full_rows = a.conv_limit / BM;
    if (a.conv_stride == 1 && !I->out_bf16 && full_rows > 0 && reinterpret_cast<uintptr_t>(a.Y) % 16 == 0) {
      const uint64_t dims[2] = {static_cast<uint64_t>(BM), static_cast<uint64_t>(full_rows)};
      const uint64_t strides[1] = {static_cast<uint64_t>(BM) * 4};
      const uint32_t box[2] = {BM, 32};
      I->tma_out = make_tmap_f32(&I->mapY, a.Y, 2, dims, strides, box) ? 1 : 0;
      I->tma_rows = static_cast<int>(full_rows);
    }
  } else if ((a.ldy * es) % 16 == 0 && reinterpret_cast<uintptr_t>(a.Y) % 16 == 0) {
    const uint64_t dims[2] = {static_cast<uint64_t>(a.rowsP), static_cast<uint64_t>(a.rowsQ)};
    const uint64_t strides[1] = {static_cast<uint64_t>(a.ldy) * es};
    const uint32_t box[2] = {BM, 32};
    I->tma_out = (I->out_bf16 ? make_tmap_bf16_plain(&I->mapY, a.Y, 2, dims, strides, box)
                              : make_tmap_f32(&I->mapY, a.Y, 2, dims, strides, box)) ? 1 : 0;
    I->tma_rows = 1 << 30;   // TMA clips ragged rows itself
    if ((a.rowsP * static_cast<int64_t>(es)) % 16) I->tma_cols = static_cast<int>(a.rowsP);
  }
  return true;
}

// K stages of all segments of a product.
static int args_stages(const GemmTcArgs& a) {
  int n = 0;
  for (int s = 0; s < a.nseg && s < 3; ++s) n += static_cast<int>(ceil_div(a.segK[s] ? a.segK[s] : a.kdim, BK));
  return n;
}

int gemm_tiles_of(const GemmInst& I) { return I.tiles_n * static_cast<int>(ceil_div(I.M, I.bn)); }

static cudaError_t set_smem_attr() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  const int bytes = static_cast<int>(kSmemBytes);
  e = cudaFuncSetAttribute(gemm_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
#if PJ_CTA_PAIRS
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
#endif
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

cudaError_t launch_gemm_tc_generic(const GemmTcArgs& a_in, int* err, int num_sms, cudaStream_t st) {
  GemmParams p;
  if (a_in.rowsQ == 0 || a_in.rowsP == 0) return cudaSuccess;
  GemmTcArgs a = a_in;
  if (!a.conv_mode)
    a.bn = single_launch_bn(a.rowsQ, ceil_div(a.rowsP, BM), args_stages(a), num_sms, a.mnQ ? 64 : 32, BN);
  const int64_t tiles_n = ceil_div(a.rowsP, BM);
  const int64_t tiles = tiles_n * ceil_div(a.rowsQ, a.bn);
  // (the expansion writes samples, which partial products could not be added into)
  const bool streamk = !a.conv_mode && !a.ex.mode && a.out_dtype != PJ_BF16 &&
                       use_stream_k(static_cast<int>(tiles), args_stages(a), num_sms);
  // CTA pairs share the Q tiles of a K-major product with an even number of tile
  // columns (half-tiles of whole 8-row swizzle atoms).
  // 256-row tiles on 2-SM MMAs wherever the tile columns pair up (gemm_cg2.cu).
  if (!streamk && gemm_cg2_eligible(a, num_sms)) return launch_gemm_cg2(a, err, num_sms, st);
  // An MN-major Q tile is bn / 64 chunks of 64 values: the pair splits the chunks.
  const bool q_pair_ok = !a.mnQ || (a.bn / 64) % 2 == 0;
  a.pair = PJ_CTA_PAIRS && !a.conv_mode && q_pair_ok && !streamk && tiles_n % 2 == 0 && a.bn % 16 == 0 &&
           num_sms >= 2;
  if (!build_gemm_inst(a, &p.single)) return cudaErrorInvalidValue;
  p.insts = nullptr;
  p.tiles = nullptr;
  p.cta_off = nullptr;
  p.num_tiles = gemm_tiles_of(p.single);
  p.err = err;
  p.stall = a.stall_stage;
  p.ex = a.ex;
  cudaError_t e = set_smem_attr();
  if (e != cudaSuccess) return e;
  int grid = p.num_tiles < num_sms ? p.num_tiles : num_sms;
  p.streamk = 0;
  if (streamk) {
    e = cudaMemset2DAsync(a.Y, a.ldy * 4, 0, a.rowsP * 4, a.rowsQ, st);
    if (e != cudaSuccess) return e;
    p.streamk = 1;
    grid = num_sms;
  }
#if PJ_CTA_PAIRS
  if (a.pair) {
    const int pairs = p.num_tiles / 2, slots = num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(2 * (pairs < slots ? pairs : slots)));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (a.mnQ || a.mnP) return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<true, true>, p);
    return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<false, true>, p);
  }
#endif
  if (a.mnP || a.mnQ)
    gemm_tc_kernel<true, false><<<grid, kThreads, kSmemBytes, st>>>(p);
  else
    gemm_tc_kernel<false, false><<<grid, kThreads, kSmemBytes, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc_grouped(const GemmInst* insts, const GemmTile* tiles, const int* cta_off, int ctas,
                                   int pair, int* err, cudaStream_t st) {
  if (ctas == 0) return cudaSuccess;
  GemmParams p;
  memset(&p.single, 0, sizeof(GemmInst));
  p.insts = insts;
  p.tiles = tiles;
  p.cta_off = cta_off;
  p.num_tiles = 0;
  p.streamk = 0;
  p.stall = -1;
  p.err = err;
  p.ex = ExpandArgs{};
  cudaError_t e = set_smem_attr();
  if (e != cudaSuccess) return e;
  if (pair) {  // CTAs 2c and 2c + 1 form a cluster; their tile lists are paired
#if !PJ_CTA_PAIRS
    return cudaErrorNotSupported;   // a build without CTA pairs plans none
#else
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(ctas));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<false, true>, p);
#endif
  }
  gemm_tc_kernel<false, false><<<ctas, kThreads, kSmemBytes, st>>>(p);  // grouped instances are K-major
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const uint16_t* Ac, const uint16_t* Bd, void* Y, int64_t ldy, int out_dtype,
                           const GemmGeom& g, int* err, int num_sms, cudaStream_t st) {
  GemmTcArgs a;
  const int64_t pitch = gemm_pitch(g);
  a.Q = Ac;
  a.ldq = pitch;
  a.rowsQ = g.M;
  a.P = Bd;
  a.ldp = pitch;
  a.rowsP = g.N;
  a.xdim = pitch;      // components are zero-padded inside each segment
  a.kdim = g.Kp_pad;
  a.Y = Y;
  a.ldy = ldy;
  a.out_dtype = out_dtype;
  if (g.nsplit == 1) {
    a.nseg = 1;
    a.segP[0] = a.segQ[0] = 0;
  } else if (!gemm_tiered(g)) {  // hi*hi + hi(A)*lo(B) + lo(A)*hi(B)
    a.nseg = 3;
    a.segQ[0] = 0;        a.segP[0] = 0;
    a.segQ[1] = 0;        a.segP[1] = g.Kp_pad;
    a.segQ[2] = g.Kp_pad; a.segP[2] = 0;
  } else {  // hi*hi over every component, then hi*lo and lo*hi over the lead ones
    const int64_t hl = g.Kp_pad, ll = g.Kp_pad + g.Kt_pad;
    a.nseg = 3;
    a.segQ[0] = 0;  a.segP[0] = 0;  a.segK[0] = g.Kp_pad;
    a.segQ[1] = hl; a.segP[1] = ll; a.segK[1] = g.Kt_pad;
    a.segQ[2] = ll; a.segP[2] = hl; a.segK[2] = g.Kt_pad;
  }
  return launch_gemm_tc_generic(a, err, num_sms, st);
}

}  // namespace pj
