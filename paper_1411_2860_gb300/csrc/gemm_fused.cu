// Fused project-then-multiply GEMM: the projection of A's groups (Sec. III-B,
// Eq. 15; here all l+1 = L = 8 projections of each group, R = block) happens in
// the GEMM kernel as A's tiles stream in, so A_c is never written to memory;
// B_d is the projected operand already in the workspace (projected once, as for
// a cached feature or weight matrix).  With the hi/lo split every component
// carries its lo term and the product keeps hi*hi + hi*lo + lo*hi.
//
// Structure: the 2-SM MMA of gemm_cg2.cu (a cluster of two CTAs computes a 256-row
// tile of B_d rows by bn rows of A; each CTA holds its 128 B_d rows and bn/2 A
// rows).  Per K chunk of 64 samples (= 64 components):
//   warp 6    loads the raw A tile (bn/2 rows x 64 samples, FP32 or BF16) by TMA
//             into a two-stage raw ring (128-byte swizzle, so the projection
//             threads read it by 16-byte chunks without bank conflicts);
//   warp 0    loads the B_d tiles (hi, and lo with the split) into the operand ring;
//   warps 7-14 project the raw tile: each thread takes (row, group) pairs, forms the
//             8 components with the kept basis (FP32 FMAs), rounds them to BF16 hi
//             (and lo = x - hi) and writes them as 16-byte chunks into the operand
//             ring's A tile in the layout the MMA reads (K-major, 128-byte swizzle);
//   warp 1    (leader) issues the 2-SM MMAs once both CTAs' B_d bytes have landed and
//             both CTAs' projection warps have arrived;
//   warps 2-5 drain the TMEM accumulator as in gemm_cg2.cu.
// With the split, the raw FP32 tile is as many bytes as the hi + lo BF16
// components it replaces, so fusing removes the A_c round trip without adding
// operand traffic; the projection's FMAs run on CUDA cores beside the MMAs.
#include <cuda_bf16.h>
#include <string.h>

#include "common.hpp"
#include "tc.cuh"
#include "tmap.hpp"
#if PJ_CTA_PAIRS
#include "tc_pair.cuh"
#endif

namespace pj {

#if PJ_CTA_PAIRS
namespace {

constexpr int FM = 128;                  // B_d rows per CTA (the pair's MMA M is 256)
constexpr int FNMAX = 256;               // most A rows per pair tile (MMA N); each CTA holds half
constexpr int FK = 64;                   // components (= samples, l+1 = L) per chunk
constexpr int kFProj = 8;                // projection warps (two per scheduler, to hide their latencies)
constexpr int kFThreads = 32 * (7 + kFProj);  // warps 0 B_d TMA, 1 MMA, 2-5 epilogue, 6 raw TMA, 7.. projection
constexpr uint32_t kFTile = 128 * FK * 2;  // one 128-row BF16 operand tile (16 KB)
constexpr uint32_t kFRaw = 2 * 128 * 128;  // one raw stage: two 128-row x 128-byte halves (FP32), one for BF16
constexpr int kFRawStages = 2;
constexpr uint32_t kFStageOut = 32 * FM * 4;

template <int NS>
constexpr int f_stages() { return NS == 1 ? 4 : 2; }
template <int NS>
constexpr size_t f_smem_bytes() {
  return 1024 + static_cast<size_t>(f_stages<NS>()) * 2 * NS * kFTile + kFRawStages * kFRaw + kFStageOut + 512;
}
static_assert(f_smem_bytes<1>() <= 232448 && f_smem_bytes<2>() <= 232448, "shared memory per block");

struct FusedParams {
  CUtensorMap mapP;     // B_d: {pitch, N} box {64, 128}, 128-byte swizzle
  CUtensorMap mapA;     // raw A: {K, M} box {64 (BF16) or 32 (FP32), bn/2}, 128-byte swizzle
  CUtensorMap mapY;     // Y: {N, M} box {128, 32}
  const float* coef;    // kept basis, Cs[t * 8 + p] = c[t, p]
  void* Y;
  int64_t ldy;
  int M, N, bn, nch;    // nch: K chunks of 64
  int64_t lo_off;       // column of B_d's lo segment (Kp_pad)
  int npp, num_pairs;
  int out_bf16, tma_cols;
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  return uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(a))) |
         (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(b))) << 16);
}

template <typename InT, int NS>
__global__ void __launch_bounds__(kFThreads, 1) gemm_fused_kernel(const __grid_constant__ FusedParams p) {
  constexpr int STAGES = f_stages<NS>();
  constexpr uint32_t kStageP = NS * kFTile, kStageQ = NS * kFTile;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_base = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw_base + 1023u) & ~1023u) - raw_base);
  uint8_t* sP = sm;
  uint8_t* sQ = sP + STAGES * kStageP;
  uint8_t* sRaw = sQ + STAGES * kStageQ;
  uint8_t* stage_out = sRaw + kFRawStages * kFRaw;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage_out + kFStageOut);
  uint64_t* full = bars;                  // [STAGES] B_d bytes of both CTAs (leader's)
  uint64_t* qready = full + STAGES;       // [STAGES] projection warps of both CTAs (leader's)
  uint64_t* empty = qready + STAGES;      // [STAGES] MMA commit, in both CTAs
  uint64_t* raw_full = empty + STAGES;    // [2] local
  uint64_t* raw_empty = raw_full + kFRawStages;
  uint64_t* acc_full = raw_empty + kFRawStages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  int* vote = reinterpret_cast<int*>(tslot + 4);
  __shared__ float s_coef[64];

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  const int qh = p.bn / 2;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&qready[s], 2 * kFProj);
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < kFRawStages; ++r) {
      mbar_init(&raw_full[r], 1);
      mbar_init(&raw_empty[r], kFProj);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 8);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 64) s_coef[threadIdx.x] = p.coef[threadIdx.x];
  if (warp == 1) {
    tmem_alloc_cg2(tslot, 512);
    tmem_relinquish_cg2();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t full_leader = mapa_shared(smem_u32(full), 0);
  const uint32_t qready_leader = mapa_shared(smem_u32(qready), 0);
  const uint32_t acc_empty_leader = mapa_shared(smem_u32(acc_empty), 0);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- B_d tiles (both CTAs), counted on the leader's stage barrier
      tma_prefetch(&p.mapP);
      int stage = 0;
      uint32_t phase = 0, last_phase[STAGES];
      bool used[STAGES];
      for (int s = 0; s < STAGES; ++s) used[s] = false;
      bool ok = true;
      for (int n = 0; ok; ++n) {
        const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
        if (pi >= p.num_pairs) break;
        const int prow = (pi % p.npp) * 2 * FM + static_cast<int>(rank) * FM;
        for (int c = 0; c < p.nch; ++c) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, p.err, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          if (leader) mbar_arrive_expect_tx(&full[stage], 2 * kStageP);
          const uint32_t bar = full_leader + stage * 8;
          tma_load_2d_cg2(sP + stage * kStageP, &p.mapP, bar, c * FK, prow);
          if (NS == 2)
            tma_load_2d_cg2(sP + stage * kStageP + kFTile, &p.mapP, bar, static_cast<int>(p.lo_off) + c * FK, prow);
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (leader)
        for (int s = 0; s < STAGES; ++s)
          if (used[s] && !mbar_wait_drain(&full[s], last_phase[s])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == 6) {
    if (lane == 0) {
      // ---------------- raw A tiles (this CTA's bn/2 rows), local ring
      tma_prefetch(&p.mapA);
      int rs = 0;
      uint32_t rph = 0, last_phase[kFRawStages];
      bool used[kFRawStages] = {false, false};
      const uint32_t bytes = (sizeof(InT) == 4 ? 2u : 1u) * static_cast<uint32_t>(qh) * 128u;
      bool ok = true;
      for (int n = 0; ok; ++n) {
        const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
        if (pi >= p.num_pairs) break;
        const int qrow = (pi / p.npp) * p.bn + static_cast<int>(rank) * qh;
        for (int c = 0; c < p.nch; ++c) {
          if (!mbar_wait(&raw_empty[rs], rph ^ 1u, p.err, DEV_TIMEOUT_RING)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&raw_full[rs], bytes);
          if (sizeof(InT) == 4) {
            tma_load_2d(sRaw + rs * kFRaw, &p.mapA, &raw_full[rs], c * FK, qrow);
            tma_load_2d(sRaw + rs * kFRaw + kFRaw / 2, &p.mapA, &raw_full[rs], c * FK + 32, qrow);
          } else {
            tma_load_2d(sRaw + rs * kFRaw, &p.mapA, &raw_full[rs], c * FK, qrow);
          }
          used[rs] = true;
          last_phase[rs] = rph;
          if (++rs == kFRawStages) {
            rs = 0;
            rph ^= 1u;
          }
        }
      }
      for (int r = 0; r < kFRawStages; ++r)
        if (used[r] && !mbar_wait_drain(&raw_full[r], last_phase[r])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp >= 7) {
    // ---------------- projection of the raw A tile into the operand ring's A tile
    const int wq = warp - 7;
    // the kept basis in registers: every item uses all 64 coefficients
    float2 cf[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
      for (int q = 0; q < 4; ++q) cf[t][q] = make_float2(s_coef[t * 8 + 2 * q], s_coef[t * 8 + 2 * q + 1]);
    int stage = 0, rs = 0;
    uint32_t phase = 0, rph = 0;
    bool ok = true;
    for (int n = 0; ok; ++n) {
      const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
      if (pi >= p.num_pairs) break;
      for (int c = 0; c < p.nch; ++c) {
        const bool w1 = mbar_wait(&raw_full[rs], rph, p.err, DEV_TIMEOUT_RING);
        const bool w2 = w1 && mbar_wait(&empty[stage], phase ^ 1u, p.err, DEV_TIMEOUT_EMPTY);
        if (!__all_sync(0xffffffffu, w1 && w2)) {
          ok = false;
          break;
        }
        const uint8_t* rawt = sRaw + rs * kFRaw;
        uint8_t* qhi = sQ + stage * kStageQ;
        // units: (8-row group, half of the 8 groups of the chunk); lane = row (lane & 7), group 4 h + (lane >> 3)
        const int units = (qh / 8) * 2;
        for (int u = wq; u < units; u += kFProj) {
          const int r = (u >> 1) * 8 + (lane & 7), h = u & 1, g = 4 * h + (lane >> 3);
          float x[8];
          if (sizeof(InT) == 4) {
            const uint8_t* row = rawt + h * (kFRaw / 2) + r * 128;
            const int c0 = 2 * (lane >> 3);
            const float4 a = *reinterpret_cast<const float4*>(row + ((c0 ^ (r & 7)) << 4));
            const float4 b = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (r & 7)) << 4));
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
          } else {
            const uint4 v = *reinterpret_cast<const uint4*>(rawt + r * 128 + ((g ^ (r & 7)) << 4));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              x[2 * k] = __uint_as_float(w[k] << 16);
              x[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
            }
          }
          // y = x C on the paired FP32 pipe: (y[2q], y[2q+1]) += x[t] (c[t,2q], c[t,2q+1])
          float2 y2[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) y2[q] = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const float2 xt = make_float2(x[t], x[t]);
#pragma unroll
            for (int q = 0; q < 4; ++q) y2[q] = __ffma2_rn(xt, cf[t][q], y2[q]);
          }
          float y[8];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            y[2 * q] = y2[q].x;
            y[2 * q + 1] = y2[q].y;
          }
          uint32_t hw[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) hw[k] = pack_bf16(y[2 * k], y[2 * k + 1]);
          const int off = r * 128 + ((g ^ (r & 7)) << 4);
          *reinterpret_cast<uint4*>(qhi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          if (NS == 2) {
            uint32_t lw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float h0 = __uint_as_float(hw[k] << 16), h1 = __uint_as_float(hw[k] & 0xffff0000u);
              lw[k] = pack_bf16(y[2 * k] - h0, y[2 * k + 1] - h1);
            }
            *reinterpret_cast<uint4*>(qhi + kFTile + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        fence_proxy_async_smem();  // the tensor core reads what these threads wrote
        __syncwarp();
        if (lane == 0) {
          mbar_arrive_cluster(qready_leader + stage * 8);
          mbar_arrive(&raw_empty[rs]);
        }
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
        if (++rs == kFRawStages) {
          rs = 0;
          rph ^= 1u;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (the leader only)
      const uint32_t idesc = idesc_bf16_f32(2 * FM, p.bn);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true, issued_any = false;
      for (int n = 0, it = 0; ok; ++n, ++it) {
        const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
        if (pi >= p.num_pairs) break;
        const int acc = it & 1;
        const uint32_t acc_phase = (it >> 1) & 1;
        if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1u, p.err, DEV_TIMEOUT_ACC_FREE)) break;
        tc_fence_after();
        const uint32_t d = tmem + acc * FNMAX;
        for (int c = 0; c < p.nch; ++c) {
          if (!mbar_wait(&full[stage], phase, p.err, DEV_TIMEOUT_FULL) ||
              !mbar_wait(&qready[stage], phase, p.err, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aP = smem_u32(sP + stage * kStageP);
          const uint32_t aQ = smem_u32(sQ + stage * kStageQ);
#pragma unroll
          for (int k = 0; k < FK / 16; ++k)
            umma_f16_cg2(d, sdesc_sw128(aP + k * 32, 0), sdesc_sw128(aQ + k * 32, 0), idesc, (c | k) != 0);
          if (NS == 2) {
#pragma unroll
            for (int k = 0; k < FK / 16; ++k)   // hi(A) x lo(B_d)
              umma_f16_cg2(d, sdesc_sw128(aP + kFTile + k * 32, 0), sdesc_sw128(aQ + k * 32, 0), idesc, 1);
#pragma unroll
            for (int k = 0; k < FK / 16; ++k)   // lo(A) x hi(B_d)
              umma_f16_cg2(d, sdesc_sw128(aP + k * 32, 0), sdesc_sw128(aQ + kFTile + k * 32, 0), idesc, 1);
          }
          issued_any = true;
          umma_commit_cg2_mc(&empty[stage], 0x3);
          if (++stage == STAGES) {
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
  } else if (warp >= 2 && warp <= 5) {
    // ---------------- epilogue (both CTAs): this CTA's 128 B_d rows of the accumulator
    const int q = warp & 3;
    const bool store_leader = warp == 2 && lane == 0;
    bool pending = false;
    for (int n = 0, it = 0;; ++n, ++it) {
      const int pi = static_cast<int>(blockIdx.x / 2) + n * static_cast<int>(gridDim.x / 2);
      if (pi >= p.num_pairs) break;
      const int ti = pi / p.npp, tj = (pi % p.npp) * 2 + static_cast<int>(rank);
      const int acc = it & 1;
      const uint32_t acc_phase = (it >> 1) & 1;
      const bool okw = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], acc_phase, p.err, DEV_TIMEOUT_ACC));
      if (lane == 0) vote[(it & 1) * 4 + q] = okw ? 1 : 0;
      named_barrier(1, 128);
      const int* v = vote + (it & 1) * 4;
      if (!(v[0] && v[1] && v[2] && v[3])) break;
      tc_fence_after();
      const int jl = q * 32 + lane;
      const int j = tj * FM + jl;
      const bool jok = j < p.N;
      for (int c0 = 0; c0 < p.bn; c0 += 32) {
        uint32_t r[32];
        tmem_ld_x32(tmem + acc * FNMAX + c0 + (static_cast<uint32_t>(q * 32) << 16), r);
        tmem_wait_ld();
        const int i0 = ti * p.bn + c0;
        if (i0 >= p.M) continue;
        if ((tj + 1) * FM <= p.tma_cols) {
          if (store_leader && pending) bulk_wait_read_all();
          named_barrier(1, 128);
          if (p.out_bf16) {
            __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(stage_out);
#pragma unroll
            for (int u = 0; u < 32; ++u) st[u * FM + jl] = __float2bfloat16_rn(__uint_as_float(r[u]));
          } else {
            float* st = reinterpret_cast<float*>(stage_out);
#pragma unroll
            for (int u = 0; u < 32; ++u) st[u * FM + jl] = __uint_as_float(r[u]);
          }
          fence_proxy_async_smem();
          named_barrier(1, 128);
          if (store_leader) {
            tma_store_2d(&p.mapY, stage_out, tj * FM, i0);
            bulk_commit_group();
            pending = true;
          }
        } else if (p.out_bf16) {
          __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(p.Y);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < p.M)
              Y[static_cast<int64_t>(i0 + u) * p.ldy + j] = __float2bfloat16_rn(__uint_as_float(r[u]));
        } else {
          float* Y = static_cast<float*>(p.Y);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (jok && i0 + u < p.M) __stcs(Y + static_cast<int64_t>(i0 + u) * p.ldy + j, __uint_as_float(r[u]));
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
  cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_cg2(tmem, 512);
  }
}

template <typename InT, int NS>
cudaError_t launch_fused_t(const FusedParams& p, int grid, cudaStream_t st) {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !done[dev]) {
    e = cudaFuncSetAttribute(gemm_fused_kernel<InT, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(f_smem_bytes<NS>()));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kFThreads);
  cfg.dynamicSmemBytes = f_smem_bytes<NS>();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gemm_fused_kernel<InT, NS>, p);
}

}  // namespace

bool gemm_fused_supported(const GemmGeom& g, int in_dtype, const void* A, int64_t lda, int num_sms) {
  const size_t es = in_dtype == PJ_F32 ? 4 : 2;
  return g.L == 8 && g.lp1 == 8 && g.compute == PJ_BF16 && !gemm_tiered(g) && g.tier == 0 && num_sms >= 2 &&
         (in_dtype == PJ_F32 || in_dtype == PJ_BF16) && reinterpret_cast<uintptr_t>(A) % 16 == 0 &&
         (lda * static_cast<int64_t>(es)) % 16 == 0 && ceil_div(g.N, FM) % 2 == 0;
}

cudaError_t launch_gemm_fused(const void* A, int64_t lda, int in_dtype, const uint16_t* Bd, const GemmGeom& g,
                              const float* Cs, void* Y, int64_t ldy, int out_dtype, int* err, int num_sms,
                              cudaStream_t st) {
  FusedParams p;
  memset(&p, 0, sizeof(p));
  const int64_t pitch = gemm_pitch(g);
  const int nch = static_cast<int>(g.Kp_pad / FK);
  const int64_t pair_cols = ceil_div(g.N, FM) / 2;
  // rows of A per pair tile: whole waves of pair tiles over the SM pairs first
  int bn = FNMAX;
  double best = 0;
  for (int b = FNMAX; b >= 64; b -= 32) {
    const int64_t tiles = ceil_div(g.M, b) * pair_cols;
    const int64_t waves = ceil_div(tiles, num_sms / 2);
    const double t = static_cast<double>(waves) * (static_cast<double>(nch) * b / 256.0 + 4.0);
    if (b == FNMAX || t < best * 0.99) {
      bn = b;
      best = t;
    }
  }
  {
    const uint64_t dims[2] = {static_cast<uint64_t>(pitch), static_cast<uint64_t>(g.N)};
    const uint64_t strides[1] = {static_cast<uint64_t>(pitch) * 2};
    const uint32_t box[2] = {FK, FM};
    if (!make_tmap_bf16(&p.mapP, Bd, 2, dims, strides, box)) return cudaErrorInvalidValue;
  }
  {
    const bool f32 = in_dtype == PJ_F32;
    const uint64_t dims[2] = {static_cast<uint64_t>(g.K), static_cast<uint64_t>(g.M)};
    const uint64_t strides[1] = {static_cast<uint64_t>(lda) * (f32 ? 4 : 2)};
    const uint32_t box[2] = {static_cast<uint32_t>(f32 ? 32 : 64), static_cast<uint32_t>(bn / 2)};
    if (!make_tmap_sw128_load(&p.mapA, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, A, 2,
                              dims, strides, box))
      return cudaErrorInvalidValue;
  }
  const size_t oes = out_dtype == PJ_BF16 ? 2 : 4;
  p.tma_cols = 1 << 30;
  if ((ldy * static_cast<int64_t>(oes)) % 16 == 0 && reinterpret_cast<uintptr_t>(Y) % 16 == 0) {
    const uint64_t dims[2] = {static_cast<uint64_t>(g.N), static_cast<uint64_t>(g.M)};
    const uint64_t strides[1] = {static_cast<uint64_t>(ldy) * oes};
    const uint32_t box[2] = {FM, 32};
    const bool okY = out_dtype == PJ_BF16 ? make_tmap_bf16_plain(&p.mapY, Y, 2, dims, strides, box)
                                          : make_tmap_f32(&p.mapY, Y, 2, dims, strides, box);
    if (!okY) return cudaErrorInvalidValue;
    // a TMA store writes the whole 16-byte chunk holding a row's last element
    if ((g.N * static_cast<int64_t>(oes)) % 16) p.tma_cols = static_cast<int>(g.N);
  } else {
    p.tma_cols = 0;   // every tile column through element stores
  }
  p.coef = Cs;
  p.Y = Y;
  p.ldy = ldy;
  p.M = static_cast<int>(g.M);
  p.N = static_cast<int>(g.N);
  p.bn = bn;
  p.nch = nch;
  p.lo_off = g.Kp_pad;
  p.npp = static_cast<int>(pair_cols);
  p.num_pairs = static_cast<int>(pair_cols * ceil_div(g.M, bn));
  p.out_bf16 = out_dtype == PJ_BF16;
  p.err = err;
  const int slots = num_sms / 2;
  const int grid = 2 * (p.num_pairs < slots ? p.num_pairs : slots);
  const bool f32 = in_dtype == PJ_F32;
  if (g.nsplit == 2)
    return f32 ? launch_fused_t<float, 2>(p, grid, st) : launch_fused_t<__nv_bfloat16, 2>(p, grid, st);
  return f32 ? launch_fused_t<float, 1>(p, grid, st) : launch_fused_t<__nv_bfloat16, 1>(p, grid, st);
}

#else   // the solo build has no CTA pairs, and the fused kernel is built on them

bool gemm_fused_supported(const GemmGeom&, int, const void*, int64_t, int) { return false; }
cudaError_t launch_gemm_fused(const void*, int64_t, int, const uint16_t*, const GemmGeom&, const float*, void*, int64_t,
                              int, int*, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

#endif

}  // namespace pj
