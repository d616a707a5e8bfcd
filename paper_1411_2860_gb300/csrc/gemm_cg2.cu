// Reduced GEMM of a single product on 2-SM MMAs (tcgen05.mma.cta_group::2):
// the same Y[i][j] = sum_k A_c[i][k] B_d[j][k] as gemm_tc.cu (the (l+1)
// smaller products of Sec. III-B, accumulated over blocks as in Eq. 2 and
// Eq. 8), with the two CTAs of a cluster acting as one 256-row MMA.
//
// Why: a CTA of gemm_tc.cu keeps its whole 128 x 256 operand pair in shared
// memory per K stage (48 KB), so four stages hold about 1 us of MMA work -- less
// than the time a TMA load from L2 takes under load on this GPU, and the tensor
// pipe waits.  In a 2-SM MMA the pair computes a 256 x N tile and each CTA holds
// only its 128 rows of P and N/2 rows of Q: 32 KB per stage, so six stages fit
// and the same shared memory covers 1.5x the MMA time.
//
// Tile: the pair takes P rows [256 c, 256 c + 256) (CTA r: its 128) and Q rows
// [bn t, bn t + bn) (CTA r loads bn/2 of them); each CTA's tensor memory holds
// the accumulator of its 128 P rows x bn Q rows, so the epilogue is the one of
// gemm_tc.cu, CTA by CTA.  The leader's (rank 0) thread issues every MMA; the
// TMA loads of both CTAs count on the leader's stage barriers, and each MMA
// commit frees the stage in both CTAs.  Both CTAs' epilogue warps arrive on the
// leader's accumulator barriers.
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

#if PJ_CTA_PAIRS
namespace {

constexpr int CM = 128;   // P rows per CTA (the pair's MMA M is 256)
constexpr int CN = 256;   // most Q rows per pair tile (MMA N); each CTA holds half
constexpr int CK = 64;
constexpr int CSTAGES = 6;
// warp 0: TMA producer; warp 1: MMA issuer (leader CTA); warps 2-9: epilogue.
// Eight epilogue warps (two per TMEM lane quadrant) split an expansion tile's
// columns in halves; the plain epilogue runs on warps 2-5.
constexpr int kCThreads = 320;
constexpr uint32_t kCStageP = CM * CK * 2;
constexpr uint32_t kCStageQ = (CN / 2) * CK * 2;
// Output staging of the TMA-store epilogue: 32 KB, four 32-column chunks of BF16
// or two of FP32 in flight, so a chunk is staged while earlier ones are stored.
constexpr uint32_t kCStageOut = 2 * 32 * CM * 4;
constexpr size_t kCSmemBytes = 1024 + CSTAGES * (kCStageP + kCStageQ) + kCStageOut + 256;
static_assert(kCSmemBytes + 64 * sizeof(float) <= 232448, "shared memory per block (dynamic + static)");

struct Cg2Params {
  GemmInst I;       // P map box {CK, CM} (MN-major: {64, CK}); Q map box {CK, bn/2} (MN-major: {64, CK})
  ExpandArgs ex;
  int npp;          // pair columns: P tile columns of 256
  int num_pairs;    // npp x Q tile rows
  int stall;        // failure-detection self-test: the producers stop after this many stages (-1: never)
  int* err;
};

template <bool kMN>
__global__ void __launch_bounds__(kCThreads, 1) gemm_cg2_kernel(const __grid_constant__ Cg2Params p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* sP = sm;
  uint8_t* sQ = sP + CSTAGES * kCStageP;
  uint8_t* stage_out = sQ + CSTAGES * kCStageQ;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage_out + kCStageOut);
  uint64_t* full = bars;
  uint64_t* empty = bars + CSTAGES;
  uint64_t* acc_full = bars + 2 * CSTAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  int* vote = reinterpret_cast<int*>(tslot + 4);   // 2 x 8 flags
  static_assert(17 * 8 + 16 + 16 * 4 <= 256, "barriers, TMEM slot and votes fit their 256 bytes");
  __shared__ float s_coef[64];
  const GemmInst* I = &p.I;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < CSTAGES; ++s) {
      mbar_init(&full[s], 1);    // the leader's expect_tx; both CTAs' copies count their bytes on it
      mbar_init(&empty[s], 1);   // the leader's MMA commit, delivered to both CTAs
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 16);  // eight epilogue warps in each CTA (the leader's is used)
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc_cg2(tslot, 512);
    tmem_relinquish_cg2();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers exist before any copy, commit or remote arrive reaches them
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t full_leader = mapa_shared(smem_u32(full), 0);
  const uint32_t acc_empty_leader = mapa_shared(smem_u32(acc_empty), 0);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs): this CTA's P rows and half of the Q rows
      tma_prefetch(&I->mapP);
      tma_prefetch(&I->mapQ);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t last_phase[CSTAGES];
      bool used[CSTAGES];
      for (int s = 0; s < CSTAGES; ++s) used[s] = false;
      bool ok = true;
      int issued = 0;
      for (int n = 0; ok; ++n) {
        const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
        if (pi >= p.num_pairs) break;
        const int pc = pi % p.npp, ti = pi / p.npp;
        const int half = I->bn / 2;
        const uint32_t stage_bytes = kCStageP + static_cast<uint32_t>(half) * CK * 2;
        const int prow = pc * 2 * CM + static_cast<int>(rank) * CM;
        for (int kk = 0; kk < I->kc; ++kk, ++issued) {
          if (issued == p.stall) {
            ok = false;
            break;
          }
          if (!mbar_wait(&empty[stage], phase ^ 1u, p.err, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          int seg = 0, kin = kk;
          if (I->ilv) {
            seg = kk % 3;
            kin = kk / 3;
          } else {
            while (seg + 1 < I->nseg && kin >= I->segKc[seg]) kin -= I->segKc[seg++];
          }
          if (leader) mbar_arrive_expect_tx(&full[stage], 2 * stage_bytes);
          const uint32_t bar = full_leader + stage * 8;
          if (kMN && I->mnP) {
            tma_load_2d_cg2(sP + stage * kCStageP, &I->mapP, bar, prow, I->segP[seg] + kin * CK);
            tma_load_2d_cg2(sP + stage * kCStageP + 8192, &I->mapP, bar, prow + 64, I->segP[seg] + kin * CK);
          } else {
            tma_load_2d_cg2(sP + stage * kCStageP, &I->mapP, bar, I->segP[seg] + kin * CK, prow);
          }
          if (kMN && I->mnQ) {
            const int hc = half / 64;
            for (int c = 0; c < hc; ++c)
              tma_load_2d_cg2(sQ + stage * kCStageQ + c * 8192, &I->mapQ, bar,
                              ti * I->bn + static_cast<int>(rank) * half + 64 * c, I->segQ[seg] + kin * CK);
          } else {
            tma_load_2d_cg2(sQ + stage * kCStageQ, &I->mapQ, bar, I->segQ[seg] + kin * CK,
                            ti * I->bn + static_cast<int>(rank) * half);
          }
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == CSTAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // The leader's barriers count both CTAs' copies: once the leader has seen every
      // issued phase complete, no copy of either CTA is still writing shared memory
      // (the peer leaves only after the cluster barrier below).
      if (leader)
        for (int s = 0; s < CSTAGES; ++s)
          if (used[s] && !mbar_wait_drain(&full[s], last_phase[s])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (the leader only)
      const bool mnP = kMN && I->mnP != 0, mnQ = kMN && I->mnQ != 0;
      const uint32_t idesc = idesc_bf16_f32(2 * CM, I->bn) | (static_cast<uint32_t>(mnP) << 15) |
                             (static_cast<uint32_t>(mnQ) << 16);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      bool issued_any = false;
      for (int n = 0, it = 0; ok; ++n, ++it) {
        const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
        if (pi >= p.num_pairs) break;
        const int acc = it & 1;
        const uint32_t acc_phase = (it >> 1) & 1;
        if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1u, p.err, DEV_TIMEOUT_ACC_FREE)) break;
        tc_fence_after();
        const uint32_t d = tmem + acc * CN;
        for (int kk = 0; kk < I->kc; ++kk) {
          if (!mbar_wait(&full[stage], phase, p.err, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aP = smem_u32(sP + stage * kCStageP);
          const uint32_t aQ = smem_u32(sQ + stage * kCStageQ);
#pragma unroll
          for (int k = 0; k < CK / 16; ++k) {
            const uint64_t dp = mnP ? sdesc_sw128_mn(aP + k * 2048, 8192) : sdesc_sw128(aP + k * 32, 0);
            const uint64_t dq = mnQ ? sdesc_sw128_mn(aQ + k * 2048, 8192) : sdesc_sw128(aQ + k * 32, 0);
            umma_f16_cg2(d, dp, dq, idesc, (kk != 0) || (k != 0));
          }
          issued_any = true;
          umma_commit_cg2_mc(&empty[stage], 0x3);
          if (++stage == CSTAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) umma_commit_cg2_mc(&acc_full[acc], 0x3);
      }
      if (issued_any) {
        umma_commit_cg2_mc(drain, 0x1);
        if (!mbar_wait_drain(drain, 0)) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
      }
    }
  } else {
    // ---------------- epilogue (both CTAs): this CTA's 128 P rows of the accumulator
    const int ew = warp - 2;   // epilogue warp 0..7
    const int q = warp & 3;    // the TMEM lane quadrant this warp may read
    const int h = ew >> 2;     // the half of an expansion tile's columns it expands
    const bool store_leader = warp == 2 && lane == 0;
    bool pending = false;
    // Everything the stores need, read from the parameters once: the stores go
    // through generic pointers, so values read through a pointer to the
    // parameters would be read again after every store.
    const ExpandArgs ex = p.ex;
    const int M = I->M, N = I->N, bn = I->bn;
    const bool out_bf16 = I->out_bf16 != 0;
    const bool tma_out = I->tma_out != 0;
    const int tma_cols = I->tma_cols;
    const int64_t ldy = I->ldy;
    void* const Yout = I->Y;
    const uint32_t chunk_bytes = 32u * CM * (out_bf16 ? 2u : 4u);
    const int nbuf = static_cast<int>(kCStageOut / chunk_bytes);
    int sbuf = 0;
    if (ex.mode)
      for (int e = threadIdx.x - 64; e < 8 * ex.lp1; e += 256) s_coef[e] = ex.coef[e];
    named_barrier(1, 256);
    for (int n = 0, it = 0;; ++n, ++it) {
      const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
      if (pi >= p.num_pairs) break;
      const int ti = pi / p.npp, tj = (pi % p.npp) * 2 + static_cast<int>(rank);
      const int acc = it & 1;
      const uint32_t acc_phase = (it >> 1) & 1;
      const bool okw = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], acc_phase, p.err, DEV_TIMEOUT_ACC));
      if (lane == 0) vote[(it & 1) * 8 + ew] = okw ? 1 : 0;
      named_barrier(1, 256);
      const int* v = vote + (it & 1) * 8;
      bool all_ok = true;
#pragma unroll
      for (int w = 0; w < 8; ++w) all_ok = all_ok && v[w] != 0;
      if (!all_ok) break;
      tc_fence_after();
      const int jl = q * 32 + lane;
      const int j = tj * CM + jl;
      const bool jok = j < N;
      if (ex.mode) {
        const int ncomp = ex.mode == 1 ? N : M;
        const int hb = bn / 2;   // a multiple of 16
        expand_tile(tmem + acc * CN + h * hb + (static_cast<uint32_t>(q * 32) << 16), hb, ex, s_coef, lane,
                    j, ncomp, ti * bn + h * hb, M, j, jok);
      }
      for (int c0 = 0; c0 < (ex.mode || h ? 0 : bn); c0 += 32) {
        uint32_t r[32];
        tmem_ld_x32(tmem + acc * CN + c0 + (static_cast<uint32_t>(q * 32) << 16), r);
        tmem_wait_ld();
        const int i0 = ti * bn + c0;
        if (i0 >= M) continue;  // uniform: no rows of this chunk exist
        if (tma_out && (tj + 1) * CM <= tma_cols) {
          // buffer sbuf was last read by the store nbuf chunks ago
          if (store_leader && pending) {
            if (nbuf == 4) bulk_wait_read_3();
            else bulk_wait_read_1();
          }
          named_barrier(2, 128);  // staging buffer free
          uint8_t* buf = stage_out + sbuf * chunk_bytes;
          if (out_bf16) {
            __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(buf);
#pragma unroll
            for (int u = 0; u < 32; ++u) st[u * CM + jl] = __float2bfloat16_rn(__uint_as_float(r[u]));
          } else {
            float* st = reinterpret_cast<float*>(buf);
#pragma unroll
            for (int u = 0; u < 32; ++u) st[u * CM + jl] = __uint_as_float(r[u]);
          }
          fence_proxy_async_smem();
          named_barrier(2, 128);  // staging written
          if (store_leader) {
            tma_store_2d(&I->mapY, buf, tj * CM, i0);
            bulk_commit_group();
            pending = true;
          }
          if (++sbuf == nbuf) sbuf = 0;
        } else if (out_bf16) {
          __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(Yout);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < M)
              Y[static_cast<int64_t>(i0 + u) * ldy + j] = __float2bfloat16_rn(__uint_as_float(r[u]));
        } else {
          float* Y = static_cast<float*>(Yout);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < M) __stcs(Y + static_cast<int64_t>(i0 + u) * ldy + j, __uint_as_float(r[u]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acc_empty_leader + acc * 8);
    }
    if (store_leader && pending) bulk_wait_all();
  }

  tc_fence_before();
  __syncthreads();
  // Neither CTA leaves while the leader's MMAs or the other CTA's copies may still
  // reach its shared or tensor memory.
  cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_cg2(tmem, 512);
  }
}

cudaError_t set_cg2_smem_attr() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  const int bytes = static_cast<int>(kCSmemBytes);
  e = cudaFuncSetAttribute(gemm_cg2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_cg2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

}  // namespace

// Rows of Q per pair tile: the height whose whole waves of pair tiles over the SM
// pairs finish first (each pair tile counted as its K stages scaled by its height
// plus a fixed cost of 4 stages); a multiple of 32 (of 128 for an MN-major Q, whose
// halves are whole 64-row chunks).
static int cg2_bn(int64_t rowsQ, int64_t pair_cols, int64_t stages, int sms, bool mnQ) {
  const int gran = mnQ ? 128 : 32;
  int best = CN;
  double best_t = 0;
  for (int bn = CN; bn >= (mnQ ? 128 : 64); bn -= gran) {
    const int64_t tiles = (rowsQ + bn - 1) / bn * pair_cols;
    const int64_t waves = (tiles + sms / 2 - 1) / (sms / 2);
    const double t = static_cast<double>(waves) * (static_cast<double>(stages) * bn / 256.0 + 4.0);
    if (bn == CN || t < best_t * 0.99) {
      best = bn;
      best_t = t;
    }
  }
  return best;
}

bool gemm_cg2_eligible(const GemmTcArgs& a, int num_sms) {
  return !a.conv_mode && num_sms >= 2 && a.rowsP > 0 && ceil_div(a.rowsP, CM) % 2 == 0;
}

static int cg2_stages(const GemmTcArgs& a) {
  int stages = 0;
  for (int s = 0; s < a.nseg && s < 3; ++s) stages += static_cast<int>(ceil_div(a.segK[s] ? a.segK[s] : a.kdim, CK));
  return stages;
}

static cudaError_t launch_cg2(Cg2Params& p, bool mn, int num_sms, cudaStream_t st) {
  cudaError_t e = set_cg2_smem_attr();
  if (e != cudaSuccess) return e;
  const int slots = num_sms / 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(2 * (p.num_pairs < slots ? p.num_pairs : slots)));
  cfg.blockDim = dim3(kCThreads);
  cfg.dynamicSmemBytes = kCSmemBytes;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (mn) return cudaLaunchKernelEx(&cfg, gemm_cg2_kernel<true>, p);
  return cudaLaunchKernelEx(&cfg, gemm_cg2_kernel<false>, p);
}

cudaError_t launch_gemm_cg2(const GemmTcArgs& a_in, int* err, int num_sms, cudaStream_t st) {
  GemmTcArgs a = a_in;
  const int64_t pair_cols = ceil_div(a.rowsP, CM) / 2;
  a.bn = cg2_bn(a.rowsQ, pair_cols, cg2_stages(a), num_sms, a.mnQ != 0);
  a.pair = 1;   // Q boxes of bn/2 rows (K-major), one CTA's half of the tile
  Cg2Params p{};
  if (!build_gemm_inst(a, &p.I)) return cudaErrorInvalidValue;
  p.npp = static_cast<int>(pair_cols);
  p.num_pairs = static_cast<int>(pair_cols * ceil_div(a.rowsQ, a.bn));
  p.stall = a.stall_stage;
  p.err = err;
  p.ex = a.ex;
  return launch_cg2(p, a.mnP || a.mnQ, num_sms, st);
}

#else   // the solo build has no CTA pairs

bool gemm_cg2_eligible(const GemmTcArgs&, int) { return false; }
cudaError_t launch_gemm_cg2(const GemmTcArgs&, int*, int, cudaStream_t) { return cudaErrorNotSupported; }

#endif

}  // namespace pj
