// Reduced cross-correlation on tcgen05 tensor cores (Sec. III-A, Eq. 11-13 with
// zero extension; all output samples).
//
// Any basis (the general path, Sec. III-A with C, D of Eq. 5-6): with
// sc_p[x] = sum_{i<L} s[x+i] c[i,p] and kd_t[g (l+1) + p] the projected template,
//   r[m][t] = sum_{g, p} sc_p[m + g L] kd_t[g (l+1) + p],
// and for the lags m = phi + L*(beta + NB*a) (phi < L, beta < NB = 64/(l+1)) the
// projected-signal sequence of phase phi, (sc_p[phi + L y])_{y, p} laid out with
// the l+1 components of a position side by side, makes every (phi, beta) the
// same Hankel product over 64-component rows as below (one row further per
// output row).  The Haar box path is the case of one component per position,
// L -> Lb phases and NB = 64; the kernel only sees PH phases and NB offsets.
//
// In the box basis of the kept Haar subspace (runs of Lb = T / R samples), the
// projected correlation is  r[m][t] = sum_{g < R} b[m + g*Lb] kb_t[g]  with
// b the projected signal and kb_t the projected template.  Splitting the lags
// as m = phi + Lb*(beta + 64*a), phi < Lb, beta < 64, turns every (phi, beta)
// into a Hankel product: output row a needs the projected-signal rows
// Row[a + c] (64 components each, c < R/64) of one phase-split row view, and
// consecutive output rows use the same rows shifted by one.
//
// Each tile computes 512 consecutive rows a0 .. a0+511 of one (phi, beta) for
// all (<= 64) templates.  The lags are paired: the MMA M side holds the
// templates twice (e = 0, 1; the e = 1 copy shifted by one 64-component
// chunk), the N side holds 256 row pairs, so one 128 x 256 MMA per 16-wide K
// step yields r at rows a0 + 2i + e.  The projected-signal rows of a tile are
// loaded once per tile into two parity rings in shared memory (the TMA splits
// even and odd rows); every K step then only re-points the UMMA descriptor by
// whole 128-byte rows.  Template chunks stream through a 4-stage pipeline;
// a separate producer warp loads the rings one tile ahead.
// TMEM holds two 128 x 256 FP32 accumulators so the epilogue of one tile
// overlaps the main loop of the next.
#include "common.hpp"
#include "tc.cuh"
#include "tmap.hpp"

namespace pj {
namespace {

constexpr int STAGES = 4;       // template-chunk stages at most (p.nst at run time)
// Warps: 0 chunk TMA, 1 UMMA, 2-5 epilogue, 6 ring TMA, and with NEPI = 2 a
// second epilogue set 7-10.
template <int NEPI>
constexpr int conv_threads() { return NEPI == 2 ? 352 : 224; }
constexpr int kRowsPerTile = 512;
constexpr uint32_t kStageA = 128 * 64 * 2;         // one template-pair chunk
constexpr int kMaxRingRows = 288;                   // per parity, Kc <= 64
constexpr uint32_t kRingParity = kMaxRingRows * 128;
constexpr uint32_t kRingBuf = 2 * kRingParity;
constexpr uint32_t kIdesc = idesc_bf16_f32(128, 256);
constexpr uint32_t kStageWarp = 2 * 16 * 32 * 4;   // one epilogue warp's staging: [2 buffers][16 rows][32 templates] FP32
// After the rings: nst template stages, then nepi x 4 warps' staging; both
// splits (4 stages + 4 warps, 3 stages + 8 warps) fill the same 80 KB.
constexpr uint32_t kChunkArea = STAGES * kStageA + 4 * kStageWarp;
static_assert(3 * kStageA + 8 * kStageWarp == kChunkArea, "the two shared-memory splits must coincide");
constexpr size_t kSmemBytes = 1024 + 2 * kRingBuf + kChunkArea + 256;

struct ConvParams {
  CUtensorMap mapTP;      // template pairs {64, (Kc+1)*128} box {64, 128}
  CUtensorMap mapG[64];   // per beta: {64, 2, NRP/2, PH} box {64, 1, RB, 1}
  CUtensorMap mapOut;     // output rows {nt, PH NB (sub), 2 (parity), npf (pairs)} box {32, 1, 1, 16}
  int tma_out;            // output rows of full row pairs go through TMA stores
  int npf;                // row pairs whose lags are valid for every (phi, beta)
  float* out;
  int64_t lags;
  int nt;
  int PH;                 // phases of the lag split (Lb for the box path, L otherwise)
  int NB;                 // row offsets beta (64 for the box path, 64 / (l+1) otherwise)
  int Kc;
  int RB;                 // rows per ring half-load
  int tiles_per_sub;
  int num_tiles;
  int nst;                // template-chunk pipeline stages (4 with one epilogue set, 3 with two)
  int pstep;              // phases computed: every pstep-th (1 = all lags)
  int* err;
};

// Tile order: the (phi, beta) sub-problem varies fastest, ordered so that
// consecutive tiles hold consecutive lags (lag offset phi + Lb * beta inside
// one row block).  Tiles running at the same time then write neighbouring
// output rows instead of rows spread over the whole output.
// With pstep > 1 only the phases phi = 0, pstep, 2 pstep, ... are computed (the
// lags m = phi + PH * u with m a multiple of pstep; PH is a multiple of pstep).
__device__ __forceinline__ void tile_coords(const ConvParams& p, int tile, int& phi, int& beta, int& a0) {
  const int nph = p.PH / p.pstep;
  const int nsub = p.NB * nph;
  const int at = tile / nsub;
  const int sub = tile - at * nsub;
  a0 = at * kRowsPerTile;
  beta = sub / nph;
  phi = (sub - beta * nph) * p.pstep;
}

template <int NEPI>
__global__ void __launch_bounds__(conv_threads<NEPI>(), 1) conv_tc_kernel(const __grid_constant__ ConvParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* ring = sm;                                  // [2 buffers][2 parities][288 rows][128 B]
  uint8_t* sA = sm + 2 * kRingBuf;                     // [STAGES][128 rows][128 B]
  float* stage = reinterpret_cast<float*>(sA + p.nst * kStageA);    // output staging
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + kChunkArea);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* ring_full = bars + 2 * STAGES;
  uint64_t* ring_empty = ring_full + 2;
  uint64_t* acc_full = ring_empty + 2;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&ring_full[a], 1);
      mbar_init(&ring_empty[a], 1);
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4 * NEPI);
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
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nchunks = p.Kc + 1;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: template chunks, one per K step
      int stage = 0;
      uint32_t phase = 0;
      uint32_t last_phase[STAGES];
      bool used[STAGES];
      for (int s = 0; s < STAGES; ++s) used[s] = false;
      bool ok = true;
      tma_prefetch(&p.mapTP);
      for (int tile = blockIdx.x; tile < p.num_tiles && ok; tile += gridDim.x) {
        for (int c = 0; c < nchunks; ++c) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, p.err, DEV_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], kStageA);
          tma_load_2d(sA + stage * kStageA, &p.mapTP, &full[stage], 0, c * 128);
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == p.nst) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      for (int s = 0; s < STAGES; ++s)
        if (used[s] && !mbar_wait_drain(&full[s], last_phase[s])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == 6) {
    if (lane == 0) {
      // ---------------- TMA producer: projected-signal rings, one tile ahead
      bool ring_used[2] = {false, false};
      uint32_t ring_last[2] = {0, 0};
      const uint32_t ring_bytes = 4u * p.RB * 128u;
      int it = 0;
      for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++it) {
        int phi, beta, a0;
        tile_coords(p, tile, phi, beta, a0);
        const int rb = it & 1;
        const uint32_t rphase = (it >> 1) & 1;
        if (!mbar_wait(&ring_empty[rb], rphase ^ 1u, p.err, DEV_TIMEOUT_RING)) break;
        mbar_arrive_expect_tx(&ring_full[rb], ring_bytes);
        for (int par = 0; par < 2; ++par)
          for (int h = 0; h < 2; ++h)
            tma_load_4d(ring + rb * kRingBuf + par * kRingParity + h * p.RB * 128, &p.mapG[beta], &ring_full[rb], 0,
                        par, a0 / 2 + h * p.RB, phi);
        ring_used[rb] = true;
        ring_last[rb] = rphase;
      }
      for (int r = 0; r < 2; ++r)
        if (ring_used[r] && !mbar_wait_drain(&ring_full[r], ring_last[r])) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- UMMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      bool ok = true;
      bool issued_any = false;
      for (int tile = blockIdx.x; tile < p.num_tiles && ok; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t bphase = (it >> 1) & 1;
        if (!mbar_wait(&acc_empty[buf], bphase ^ 1u, p.err, DEV_TIMEOUT_ACC_FREE)) break;
        if (!mbar_wait(&ring_full[buf], bphase, p.err, DEV_TIMEOUT_RING)) break;
        tc_fence_after();
        const uint32_t d = tmem + buf * 256;
        const uint32_t ring0 = smem_u32(ring + buf * kRingBuf);
        for (int c = 0; c < nchunks; ++c) {
          if (!mbar_wait(&full[stage], phase, p.err, DEV_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aA = smem_u32(sA + stage * kStageA);
          // rows a0 + 2i + c for i < 256: parity (c & 1), ring row (c >> 1) + i
          const uint32_t aB = ring0 + (c & 1) * kRingParity + (c >> 1) * 128;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            umma_f16(d, sdesc_sw128(aA + k * 32, 0), sdesc_sw128(aB + k * 32, 0), kIdesc, (c | k) != 0);
          issued_any = true;
          umma_commit(&empty[stage]);
          if (++stage == p.nst) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) {
          umma_commit(&ring_empty[buf]);
          umma_commit(&acc_full[buf]);
        }
      }
      // Commit only behind issued MMAs: a commit with nothing to track is never issued.
      if (issued_any) {
        umma_commit(drain);
        if (!mbar_wait_drain(drain, 0)) atomicCAS(p.err, 0, DEV_TIMEOUT_DRAIN);
      }
    }
  } else if ((warp >= 2 && warp <= 5) || (NEPI == 2 && warp >= 7)) {
    // ---------------- epilogue: warp q drains TMEM lanes 32q .. 32q+31, i.e. the
    // output rows of parity e = q / 2 for templates t0 .. t0+31, column = row pair;
    // with two sets, set 0 (warps 2-5) takes the even 32-column chunks and set 1
    // (warps 7-10) the odd ones.
    // Full row pairs leave through the warp's own TMA bulk stores of 16 rows x
    // 32 templates from two alternating 2 KB staging buffers, so a buffer is
    // only waited for when the store issued two before it still reads it, and
    // the four warps never wait for one another.  Ragged rows: direct stores.
    const int q = warp & 3;
    const int set = warp >= 7 ? 1 : 0;
    const int e = q >> 1;
    const int t0 = (q & 1) * 32;
    const int t = t0 + lane;
    const bool tok = t < p.nt;
    const bool wlive = t0 < p.nt;
    float* stg = stage + (set * 4 + q) * 2 * 16 * 32;   // [2 buffers][16 rows][32 templates]
    bool issued = false;
    int it = 0;
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++it) {
      int phi, beta, a0;
      tile_coords(p, tile, phi, beta, a0);
      const int buf = it & 1;
      const uint32_t bphase = (it >> 1) & 1;
      // Uniform outcome across the warp, so no lane is left alone at a __syncwarp.
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], bphase, p.err, DEV_TIMEOUT_ACC))) break;
      tc_fence_after();
      // lag of column i: phi + PH * (beta + NB * (a0 + 2i + e))
      const int64_t m0 = phi + static_cast<int64_t>(p.PH) * (beta + static_cast<int64_t>(p.NB) * (a0 + e));
      const int64_t dm = static_cast<int64_t>(p.PH) * 2 * p.NB;
      const int sub = beta * p.PH + phi;
      for (int c0 = 32 * set; c0 < 256; c0 += 32 * NEPI) {
        if (m0 + dm * c0 >= p.lags) break;  // this and every later column lies past the last lag
        uint32_t r[32];
        tmem_ld_x32(tmem + buf * 256 + c0 + (static_cast<uint32_t>(q * 32) << 16), r);
        tmem_wait_ld();
        const int pair0 = a0 / 2 + c0;
        if (p.tma_out && pair0 + 32 <= p.npf) {
          if (wlive) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              float* sb = stg + hh * 16 * 32;
              if (lane == 0) bulk_wait_read_1();  // the store that last read buffer hh is done
              __syncwarp();
#pragma unroll
              for (int u = 0; u < 16; ++u) sb[u * 32 + lane] = __uint_as_float(r[hh * 16 + u]);
              fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0) {
                tma_store_4d(&p.mapOut, sb, t0, sub, e, pair0 + hh * 16);
                bulk_commit_group();
                issued = true;
              }
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int64_t m = m0 + dm * (c0 + u);
            if (tok && m < p.lags) __stcs(p.out + m * p.nt + t, __uint_as_float(r[u]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (lane == 0 && issued) bulk_wait_all();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Reductions of 16 chunks or more (R >= 1024) keep the MMA busy: four template
// stages and one epilogue set.  Shorter ones are bound by the output write and
// drain the accumulators with two epilogue sets (three template stages).
int conv_epilogue_sets(int Kc) { return Kc >= 16 ? 1 : 2; }

}  // namespace

// Tensor maps depend only on the workspace buffers and the geometry; encoding
// 65 of them costs tens of microseconds of host time, so the last few are
// kept per host thread and reused while (G, TP, geometry) repeat.
struct ConvMapCache {
  const void* G = nullptr;
  const void* TP = nullptr;
  int64_t S = -1, T = -1, nt = -1, R = -1;
  int L = -1, box = -1;
  ConvParams p;
};

cudaError_t launch_conv_tc(const uint16_t* G, const uint16_t* TP, float* out, const ConvGeom& g, int* err,
                           int num_sms, cudaStream_t st, int pstep) {
  static thread_local ConvMapCache cache[4];
  static thread_local int next_slot = 0;
  ConvMapCache* hit = nullptr;
  for (auto& c : cache)
    if (c.G == G && c.TP == TP && c.S == g.S && c.T == g.T && c.nt == g.nt && c.R == g.R && c.L == g.L &&
        c.box == g.box)
      hit = &c;
  if (!hit) {
    hit = &cache[next_slot];
    next_slot = (next_slot + 1) % 4;
    hit->G = nullptr;  // invalid until every map is built
    ConvParams& p = hit->p;
    {
      const uint64_t dims[2] = {64, static_cast<uint64_t>(g.Kc + 1) * 128};
      const uint64_t strides[1] = {128};
      const uint32_t box[2] = {64, 128};
      if (!make_tmap_bf16(&p.mapTP, TP, 2, dims, strides, box)) return cudaErrorInvalidValue;
    }
    const int NY = 256 + (g.Kc >> 1);
    const int RB = static_cast<int>(round_up(ceil_div(NY, 2), 8));
    // Row view of (phi, beta): position beta of every phase row, in the copy shifted by
    // sigma = beta mod ncopy positions, so that it starts on a 16-byte boundary.
    for (int beta = 0; beta < g.NB; ++beta) {
      const int sigma = beta % g.ncopy;
      const int64_t off = static_cast<int64_t>(beta - sigma) * g.lp1c;
      const uint16_t* base = G + static_cast<int64_t>(sigma) * g.PH * g.P + off;
      const uint64_t dims[4] = {64, 2, static_cast<uint64_t>(g.NRP / 2), static_cast<uint64_t>(g.PH)};
      const uint64_t strides[3] = {128, 256, static_cast<uint64_t>(g.P) * 2};
      const uint32_t box[4] = {64, 1, static_cast<uint32_t>(RB), 1};
      if (!make_tmap_bf16(&p.mapG[beta], base, 4, dims, strides, box)) return cudaErrorInvalidValue;
    }
    p.lags = g.lags;
    p.nt = static_cast<int>(g.nt);
    p.PH = g.PH;
    p.NB = g.NB;
    p.Kc = g.Kc;
    p.RB = RB;
    p.tiles_per_sub = g.tiles_per_sub;
    p.num_tiles = static_cast<int>(g.tiles_per_sub * g.per);
    p.nst = conv_epilogue_sets(g.Kc) == 1 ? 4 : 3;
    hit->TP = TP;
    hit->S = g.S;
    hit->T = g.T;
    hit->nt = g.nt;
    hit->R = g.R;
    hit->L = g.L;
    hit->box = g.box;
    hit->G = G;
  }
  ConvParams& p = hit->p;
  p.out = out;
  p.err = err;
  p.pstep = pstep;
  p.num_tiles = static_cast<int>(g.tiles_per_sub * g.NB * (g.PH / pstep));
  // Output map for the TMA-store epilogue: rows of full row pairs, every (phi, beta).
  const int64_t a_full = g.lags / g.per;
  p.npf = static_cast<int>(a_full / 2);
  p.tma_out = 0;
  if (g.nt % 4 == 0 && p.npf > 0) {
    const uint64_t rowb = static_cast<uint64_t>(g.nt) * 4;
    const uint64_t dims[4] = {static_cast<uint64_t>(g.nt), static_cast<uint64_t>(g.per), 2,
                              static_cast<uint64_t>(p.npf)};
    const uint64_t strides[3] = {rowb, rowb * g.per, rowb * 2 * g.per};
    const uint32_t box[4] = {32, 1, 1, 16};
    p.tma_out = make_tmap_f32(&p.mapOut, out, 4, dims, strides, box) ? 1 : 0;
  }
  const int nepi = conv_epilogue_sets(g.Kc);
  static bool attr_set[2][64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[nepi - 1][dev]) {
    e = cudaFuncSetAttribute(nepi == 2 ? conv_tc_kernel<2> : conv_tc_kernel<1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemBytes));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[nepi - 1][dev] = true;
  }
  const int grid = p.num_tiles < num_sms ? p.num_tiles : num_sms;
  if (nepi == 2)
    conv_tc_kernel<2><<<grid, conv_threads<2>(), kSmemBytes, st>>>(p);
  else
    conv_tc_kernel<1><<<grid, conv_threads<1>(), kSmemBytes, st>>>(p);
  return cudaGetLastError();
}

// Lags between computed ones (every step-th lag): linear interpolation of the
// two computed neighbours, the nearest computed lag past the last one.  A row
// of nt templates is handled by lpr lanes (the smallest power of two covering
// the row four templates at a time when rows are 16-byte aligned), so a warp
// fills 32 / lpr missing lags.
__global__ void __launch_bounds__(256) conv_interp_kernel(float* __restrict__ out, int64_t lags, int nt, int step,
                                                          int64_t rows, int lpr) {
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t q = gt / lpr;
  const int lane = static_cast<int>(gt - q * lpr);
  if (q >= rows) return;
  const uint32_t per = static_cast<uint32_t>(step - 1);
  const int64_t grp = static_cast<int64_t>(static_cast<uint64_t>(q) / per);
  const int64_t m0 = grp * step;
  const int64_t m = m0 + (q - grp * per) + 1;
  if (m >= lags) return;
  const int64_t m1 = m0 + step;
  const bool has1 = m1 < lags;
  const float w1 = has1 ? static_cast<float>(m - m0) / static_cast<float>(step) : 0.0f;
  const float w0 = has1 ? static_cast<float>(m1 - m) / static_cast<float>(step) : 1.0f;
  const float* r0 = out + m0 * nt;
  const float* r1 = out + (has1 ? m1 : m0) * nt;
  float* o = out + m * nt;
  if ((nt & 3) == 0) {
    for (int c = lane; c < nt / 4; c += lpr) {
      const float4 a = reinterpret_cast<const float4*>(r0)[c];
      const float4 b = reinterpret_cast<const float4*>(r1)[c];
      reinterpret_cast<float4*>(o)[c] =
          make_float4(w0 * a.x + w1 * b.x, w0 * a.y + w1 * b.y, w0 * a.z + w1 * b.z, w0 * a.w + w1 * b.w);
    }
  } else {
    for (int c = lane; c < nt; c += lpr) o[c] = w0 * r0[c] + w1 * r1[c];
  }
}

cudaError_t launch_conv_interp(float* out, const ConvGeom& g, int step, cudaStream_t st) {
  if (step <= 1) return cudaSuccess;
  const int64_t rows = ceil_div(g.lags, step) * (step - 1);
  if (rows == 0) return cudaSuccess;
  const int64_t per_row = g.nt % 4 == 0 ? g.nt / 4 : g.nt;
  int lpr = 1;
  while (lpr < 32 && lpr < per_row) lpr *= 2;
  conv_interp_kernel<<<static_cast<unsigned>(ceil_div(rows * lpr, 256)), 256, 0, st>>>(
      out, g.lags, static_cast<int>(g.nt), step, rows, lpr);
  return cudaGetLastError();
}

}  // namespace pj
