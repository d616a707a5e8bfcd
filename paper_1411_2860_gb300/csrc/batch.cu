// Batched launch: many uneven projected GEMM and CONV instances in a handful
// of kernels -- four batched projection launches and ONE persistent grouped
// tcgen05 GEMM over the tiles of every instance.
//
// GEMM instances are the projected products of Sec. III-B.  A correlation
// instance (valid cross-correlation with the box/Haar projection, Sec. III-A,
// Eq. 11-13) is lowered to GEMMs, one per (phase, template): with the
// projected signal b^phi viewed as rows of 128 samples and the projected
// template kb in a 128 x (R + 127) Toeplitz matrix Kt[p][j] = kb[j - p],
//   r[phi + Lb (128 i + p)] = sum_j b^phi[128 i + j] Kt[p][j],
// i.e. output row i of the GEMM holds 128 consecutive lags of that phase.
// The signal operand is read in the row-split mode of the grouped GEMM (chunk
// k of row i = view row i + k/2, half k mod 2), so nothing is materialised
// per lag; the Toeplitz matrix of each template is built once per run.
// GEMM instances with E4M3 compute are quantised after the projections and
// multiplied by a second persistent grouped launch of the block-scaled kernel.
//
// The plan is tuned on the host: each GEMM instance gets a tile height that
// covers its rows with the least padding, long reduced dimensions may be cut
// into pieces (by a cost model) whose partial products are added into the
// (zeroed) FP32 output, and the tiles are dealt to the persistent CTAs sorted
// by reduced length, round-robin (or, as an option, longest first onto the
// least-loaded CTA).  By default the BF16 tiles go to clusters of two CTAs in
// pairs that share their A_c tiles (see schedule_kind).  The cost model's
// constants, the height policy, the largest split, the order and the pairing
// are knobs (pj_batch_tuning) that a measuring autotuner can search.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "common.hpp"
#include "mx.cuh"
#include "tc.cuh"

struct pj_batch_plan;

namespace pj {
namespace {

struct SigJob {
  const float* s;
  uint16_t* Q;
  uint16_t* Qlo;     // residual rows of the split, or NULL
  int64_t S, n, block0;
  int Lb, phi;
  float scale;
};

struct TplJob {
  const float* k;
  uint16_t* Kt;
  int64_t R, Kpad, ldk, block0;  // row p: hi at [0, Kpad), split residual at [Kpad, 2 Kpad)
  int Lb, nsplit;
  float scale;
};


__device__ __forceinline__ uint16_t to_bf16(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float from_bf16(uint16_t b) { return __uint_as_float(uint32_t(b) << 16); }

// One phase of a projected signal: Q[u] = b[phi + Lb u], b[x] = sum_{v<Lb} s[x+v] / sqrt(Lb);
// with the split, Qlo[u] = bf16(b - Q[u]).
__global__ void __launch_bounds__(256) batch_signal_kernel(const SigJob* __restrict__ jobs,
                                                           const int* __restrict__ job_of) {
  const SigJob& J = jobs[job_of[blockIdx.x]];
  const int64_t u = (static_cast<int64_t>(blockIdx.x) - J.block0) * blockDim.x + threadIdx.x;
  if (u >= J.n) return;
  const int64_t x = J.phi + static_cast<int64_t>(J.Lb) * u;
  float v = 0.0f;
  if (x + J.Lb <= J.S) {
    for (int w = 0; w < J.Lb; ++w) v += __ldg(J.s + x + w);
    v *= J.scale;
  }
  const uint16_t h = to_bf16(v);
  J.Q[u] = h;
  if (J.Qlo) J.Qlo[u] = to_bf16(v - from_bf16(h));
}

// Toeplitz matrix of one projected template: Kt[p][j] = kb[j - p], kb[g] = sum_{v<Lb} k[g Lb + v] / sqrt(Lb);
// with the split, Kt[p][Kpad + j] = bf16(kb[j - p] - Kt[p][j]).
__global__ void __launch_bounds__(256) batch_toeplitz_kernel(const TplJob* __restrict__ jobs,
                                                             const int* __restrict__ job_of) {
  const TplJob& J = jobs[job_of[blockIdx.x]];
  const int64_t e = (static_cast<int64_t>(blockIdx.x) - J.block0) * blockDim.x + threadIdx.x;
  if (e >= 128 * J.Kpad) return;
  const int64_t p = e / J.Kpad, jj = e - p * J.Kpad;
  const int64_t g = jj - p;
  float v = 0.0f;
  if (g >= 0 && g < J.R) {
    for (int w = 0; w < J.Lb; ++w) v += __ldg(J.k + g * J.Lb + w);
    v *= J.scale;
  }
  const uint16_t h = to_bf16(v);
  J.Kt[p * J.ldk + jj] = h;
  if (J.nsplit > 1) J.Kt[p * J.ldk + J.Kpad + jj] = to_bf16(v - from_bf16(h));
}

// E4M3 lowered correlation.  The phase's BF16 hi + lo sequence is quantised per
// block of 32 (scale 2^e from the block's amax, mx.cuh), one thread per block;
// then the block scales are laid out per GEMM tile and K stage as the
// block-scaled MMA reads them: tile row i of stage k reads Q row
// r = t bn + i + k, whose K block b is signal block 4 r + b (the overlapping
// windows of the lowering share their blocks, so one scale per block serves
// every row that reads it).
struct SigQJob {
  const uint16_t* Q;
  const uint16_t* Qlo;
  uint8_t* QE;       // E4M3 sequence, q_rows x 128
  uint8_t* bsc;      // UE8M0 scale of each block of 32
  int64_t nblk, block0;
};

struct SfExpJob {
  const uint8_t* bsc;
  uint8_t* sf;        // per tile and stage: 1024 bytes
  int64_t q_rows, total, block0;   // total = tiles x kc x bn x 4 scale bytes
  int kc, bn;
};

__global__ void __launch_bounds__(256) batch_sigquant_kernel(const SigQJob* __restrict__ jobs,
                                                             const int* __restrict__ job_of) {
  const SigQJob& J = jobs[job_of[blockIdx.x]];
  const int64_t blk = (static_cast<int64_t>(blockIdx.x) - J.block0) * blockDim.x + threadIdx.x;
  if (blk >= J.nblk) return;
  float x[32];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint4 h = reinterpret_cast<const uint4*>(J.Q + blk * 32)[v];
    const uint4 l = reinterpret_cast<const uint4*>(J.Qlo + blk * 32)[v];
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      x[8 * v + 2 * w] = from_bf16(static_cast<uint16_t>(hw[w] & 0xFFFFu)) +
                         from_bf16(static_cast<uint16_t>(lw[w] & 0xFFFFu));
      x[8 * v + 2 * w + 1] = from_bf16(static_cast<uint16_t>(hw[w] >> 16)) +
                             from_bf16(static_cast<uint16_t>(lw[w] >> 16));
    }
  }
  float am = 0.0f;
#pragma unroll
  for (int k = 0; k < 32; ++k) am = fmaxf(am, fabsf(x[k]));
  const int e = mx_exponent(am);
  const float inv = ldexpf(1.0f, -e);
  uint32_t q[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    q[k] = e4m3x2(x[4 * k], x[4 * k + 1], inv) | (e4m3x2(x[4 * k + 2], x[4 * k + 3], inv) << 16);
  reinterpret_cast<uint4*>(J.QE + blk * 32)[0] = make_uint4(q[0], q[1], q[2], q[3]);
  reinterpret_cast<uint4*>(J.QE + blk * 32)[1] = make_uint4(q[4], q[5], q[6], q[7]);
  J.bsc[blk] = static_cast<uint8_t>(e + 127);
}

__global__ void __launch_bounds__(256) batch_sfexpand_kernel(const SfExpJob* __restrict__ jobs,
                                                             const int* __restrict__ job_of) {
  const SfExpJob& J = jobs[job_of[blockIdx.x]];
  const int64_t e = (static_cast<int64_t>(blockIdx.x) - J.block0) * blockDim.x + threadIdx.x;
  if (e >= J.total) return;
  const int b = static_cast<int>(e & 3);
  const int64_t rest = e >> 2;
  const int i = static_cast<int>(rest % J.bn);
  const int64_t tk = rest / J.bn;             // tile t, stage k: t * kc + k
  const int64_t r = (tk / J.kc) * J.bn + i + tk % J.kc;
  const uint8_t v = r < J.q_rows ? J.bsc[4 * r + b] : static_cast<uint8_t>(127);
  const int atom = i >> 7, ar = i & 127;
  J.sf[(tk * 2 + atom) * 512 + (ar & 31) * 16 + (ar >> 5) * 4 + b] = v;
}

// Zeroes the FP32 output of an instance whose reduced dimension is split.
struct ZeroJob {
  float* Y;
  int64_t rows, cols, ld, block0;
};

__global__ void __launch_bounds__(256) batch_zero_kernel(const ZeroJob* __restrict__ jobs,
                                                         const int* __restrict__ job_of) {
  const ZeroJob& J = jobs[job_of[blockIdx.x]];
  const int64_t r0 = (static_cast<int64_t>(blockIdx.x) - J.block0) * 4;
  for (int64_t r = r0; r < r0 + 4 && r < J.rows; ++r)
    for (int64_t c = threadIdx.x; c < J.cols; c += blockDim.x) J.Y[r * J.ld + c] = 0.0f;
}

}  // namespace
}  // namespace pj

using namespace pj;

struct pj_batch_plan {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  TmaJob* d_tma_jobs[kTmaClasses] = {};
  int4* d_tma_units[kTmaClasses] = {};
  int64_t tma_units[kTmaClasses] = {};
  RowsJob* d_rows[kProjectionClasses] = {};
  ColsJob* d_cols[kProjectionClasses] = {};
  SigJob* d_sig = nullptr;
  TplJob* d_tpl = nullptr;
  int n_rows[kProjectionClasses] = {}, n_cols[kProjectionClasses] = {}, n_sig = 0, n_tpl = 0;
  // block -> job tables of the job-table launches
  int* rows_of[kProjectionClasses] = {};
  int* cols_of[kProjectionClasses] = {};
  int* sig_of = nullptr;
  int* tpl_of = nullptr;
  int64_t rows_blocks[kProjectionClasses] = {}, cols_blocks[kProjectionClasses] = {}, sig_blocks = 0, tpl_blocks = 0;
  SigQJob* d_sigq = nullptr;   // E4M3 correlations: signal quantisation and scale layout
  SfExpJob* d_sfx = nullptr;
  int* sigq_of = nullptr;
  int* sfx_of = nullptr;
  int64_t sigq_blocks = 0, sfx_blocks = 0;
  GemmInst* d_insts = nullptr;
  GemmTile* d_tiles = nullptr;
  int* d_cta_off = nullptr;
  int ctas = 0;
  int paired = 0;        // BF16 launch in clusters of two CTAs
  MxInst* d_mx = nullptr;
  GemmTile* d_mx_tiles = nullptr;
  int* d_mx_cta_off = nullptr;
  int mx_ctas = 0;
  MxQuantSide* d_qsides = nullptr;
  int* qsides_of = nullptr;
  int64_t qsides_blocks = 0;
  ZeroJob* d_zero = nullptr;
  int* zero_of = nullptr;
  int64_t zero_blocks = 0;
  int sms = 0;
  pj_batch_info info{};
};

namespace {

constexpr int kMaxCtas = 1024;  // persistent CTAs of one grouped launch (at most one per SM)

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  }
};

// A TMA projection job before its tensor map is encoded.
struct TmaSpec {
  const void* X;
  int64_t ld;
  int in_dtype, cols;
  GemmGeom g{};
  const float* coef;
  uint16_t* out;
  int quant = 0;          // E4M3 output (classes +16): components and scales as q says
  MxQuantSide q{};
  int bulk = 0;           // rows read by bulk copies (classes +32)
};
inline int tma_class(int in_dtype, int lp1) { return (in_dtype == PJ_BF16 ? 8 : 0) + lp1 - 1; }

// Resolved tuning knobs (pj_batch_tuning with the defaults filled in).
struct Tuning {
  int schedule = 0, tile_rows = 0, max_split = 16, solo = 0;
  double t_tile = 0.8, t_stage = 0.34, t_out_kb = 0.02;
};

pj_status resolve_tuning(const pj_batch_tuning* t, Tuning* out) {
  Tuning r;
  if (t) {
    if (t->schedule < 0 || t->schedule > 2) return fail(PJ_EINVAL, "tuning.schedule must be 0, 1 or 2");
    if (t->tile_rows != 0 && (t->tile_rows < 32 || t->tile_rows > 256 || t->tile_rows % 32))
      return fail(PJ_EINVAL, "tuning.tile_rows must be 0 or a multiple of 32 in [32, 256]");
    if (t->max_split < 0 || t->max_split > 64) return fail(PJ_EINVAL, "tuning.max_split must be in [0, 64]");
    if (t->solo != 0 && t->solo != 1) return fail(PJ_EINVAL, "tuning.solo must be 0 or 1");
    if (t->us_per_tile < 0 || t->us_per_stage < 0 || t->us_per_out_kb < 0)
      return fail(PJ_EINVAL, "tuning costs must be >= 0");
    r.schedule = t->schedule;
    r.tile_rows = t->tile_rows;
    r.solo = t->solo;
    if (t->max_split) r.max_split = t->max_split;
    if (t->us_per_tile > 0) r.t_tile = t->us_per_tile;
    if (t->us_per_stage > 0) r.t_stage = t->us_per_stage;
    if (t->us_per_out_kb > 0) r.t_out_kb = t->us_per_out_kb;
  }
  if (r.schedule == 1) r.max_split = 1;
  *out = r;
  return PJ_OK;
}

// Rows of A_c per tile: the fixed height, or the fewest tiles of at most bnmax
// rows with the least padding (granularity gran).
int pick_bn(int64_t M, int gran, int bnmax, const Tuning& t) {
  if (t.tile_rows) {
    int b = t.tile_rows < bnmax ? t.tile_rows : bnmax;
    b -= b % gran;
    return b < gran ? gran : b;
  }
  const int64_t tiles = ceil_div(M > 0 ? M : 1, bnmax);
  const int64_t b = round_up(ceil_div(M > 0 ? M : 1, tiles), gran);
  return static_cast<int>(b < bnmax ? b : bnmax);
}

// The largest split the tuner may give an instance: FP32 output, >= 8 K stages a piece.
int split_cap(int64_t stages, bool fp32_out, const Tuning& t) {
  if (!fp32_out || t.max_split <= 1) return 1;
  int s = 1;
  while (s * 2 <= t.max_split && stages / (s * 2) >= 8) s *= 2;
  return s;
}

// One GEMM of the grouped launches, before tiling.
struct GemmPlanned {
  int kind;             // 0 = BF16 kernel, 1 = E4M3 kernel
  int index;            // into Built::gemms or Built::mx
  int tiles_m, tiles_n; // tile rows (of bn A_c rows) and columns (of 128 B_d rows)
  int stages;           // K stages of a whole tile
  int bn, cap;          // tile height, largest split
  bool out_bf16;
};

struct Built {
  Tuning tune;
  std::vector<MxGemmArgs> mx;
  std::vector<MxQuantSide> qsides;
  std::vector<ZeroJob> zeros;
  std::vector<GemmPlanned> planned;
  size_t mx_off = 0, mx_tiles_off = 0, mx_cta_off = 0, cta_off_off = 0, qsides_off = 0, qsides_map_off = 0,
         zero_off = 0, zero_map_off = 0;
  int64_t qsides_total = 0, zero_total = 0;
  int tiles_cap = 0, mx_tiles_cap = 0;
  std::vector<TmaSpec> tma[kTmaClasses];
  int64_t tma_units[kTmaClasses] = {};
  size_t tma_jobs_off[kTmaClasses] = {}, tma_units_off[kTmaClasses] = {};
  std::vector<RowsJob> rows[kProjectionClasses];
  std::vector<ColsJob> cols[kProjectionClasses];
  std::vector<SigJob> sig;
  std::vector<TplJob> tpl;
  std::vector<SigQJob> sigq;
  std::vector<SfExpJob> sfx;
  size_t sigq_off = 0, sfx_off = 0, sigq_map_off = 0, sfx_map_off = 0;
  int64_t sigq_total = 0, sfx_total = 0;
  std::vector<GemmTcArgs> gemms;
  std::vector<std::tuple<int, int, int, const double*>> bases;  // kind, L, lp1, user matrix
  size_t basis_off = 0, rows_off[kProjectionClasses] = {}, cols_off[kProjectionClasses] = {};
  size_t sig_off = 0, tpl_off = 0, insts_off = 0, tiles_off = 0;
  size_t rows_map_off[kProjectionClasses] = {}, cols_map_off[kProjectionClasses] = {}, sig_map_off = 0,
         tpl_map_off = 0;
  int64_t rows_total[kProjectionClasses] = {}, cols_total[kProjectionClasses] = {}, sig_total = 0, tpl_total = 0;
  size_t total = 0;
};

template <typename T>
T* ptr(void* ws, size_t off) {
  return ws ? reinterpret_cast<T*>(static_cast<char*>(ws) + off) : nullptr;
}

// Walks the descriptors, validates them and lays out the workspace.  With
// ws == nullptr only the sizes are computed.
pj_status layout(const pj_batch_desc* d, int n, const pj_batch_tuning* tuning, void* ws, Built* out) {
  if (!d || n < 1) return fail(PJ_EINVAL, "batch needs at least one descriptor");
  Built& b = *out;
  PJ_TRY(resolve_tuning(tuning, &b.tune));
  Layout L;
  L.take(kHeaderBytes);
  // distinct GEMM bases, each with its own basis area
  std::map<std::tuple<int, int, int, const double*>, int> basis_index;
  std::vector<GemmGeom> gg(n);
  std::vector<ConvGeom> cg(n);
  for (int i = 0; i < n; ++i) {
    const pj_batch_desc& x = d[i];
    if (x.op == PJ_OP_GEMM && x.prec.compute != PJ_BF16 && x.prec.compute != PJ_E4M3)
      return fail(PJ_EUNSUPPORTED, "batch entry %d: GEMM compute PJ_BF16 or PJ_E4M3", i);
    if (x.op == PJ_OP_CONV && x.prec.compute != PJ_BF16 && x.prec.compute != PJ_E4M3)
      return fail(PJ_EUNSUPPORTED, "batch entry %d: correlations compute in PJ_BF16 or PJ_E4M3", i);
    if (x.op == PJ_OP_CONV && x.prec.compute == PJ_E4M3 && x.prec.split_terms != 1)
      return fail(PJ_EUNSUPPORTED,
                  "batch entry %d: E4M3 correlations take split_terms = 1 (the residual of the lowered "
                  "signal would be a second sequence, which the product's row segments cannot address)", i);
    if (x.prec.split_lead) return fail(PJ_EUNSUPPORTED, "batch entry %d: split_lead must be 0 in a batch", i);
    if (x.prec.fp8_tier) return fail(PJ_EUNSUPPORTED, "batch entry %d: fp8_tier must be 0 in a batch", i);
    if (x.op == PJ_OP_GEMM) {
      PJ_TRY(gemm_geom(x.M, x.N, x.K, x.block, x.R, &x.basis, &x.prec, &gg[i]));
      if (x.in_dtype != PJ_F32 && x.in_dtype != PJ_BF16)
        return fail(PJ_EUNSUPPORTED, "batch entry %d: GEMM input PJ_F32 or PJ_BF16", i);
      if (x.out_dtype != PJ_F32 && x.out_dtype != PJ_BF16)
        return fail(PJ_EUNSUPPORTED, "batch entry %d: GEMM output PJ_F32 or PJ_BF16", i);
      if (x.M > 0 && x.K > 0 && (!x.A || x.lda < x.K)) return fail(PJ_EINVAL, "batch entry %d: bad A / lda", i);
      if (x.K > 0 && x.N > 0 && (!x.B || x.ldb < x.N)) return fail(PJ_EINVAL, "batch entry %d: bad B / ldb", i);
      if (x.M > 0 && x.N > 0 && (!x.Y || x.ldy < x.N)) return fail(PJ_EINVAL, "batch entry %d: bad Y / ldy", i);
      if (x.K == 0) return fail(PJ_EUNSUPPORTED, "batch entry %d: K = 0", i);
      auto key = std::make_tuple(x.basis.kind, x.basis.L, gg[i].lp1, x.basis.user_C);
      if (!basis_index.count(key)) {
        const int id = static_cast<int>(b.bases.size());
        basis_index[key] = id;
        b.bases.push_back(key);
      }
    } else if (x.op == PJ_OP_CONV) {
      // The split (hi + lo residual, three reduced products) is carried by the
      // grouped GEMM; the geometry is that of the plain correlation.
      if (x.prec.split_terms != 1 && x.prec.split_terms != 2)
        return fail(PJ_EUNSUPPORTED, "batch entry %d: split_terms must be 1 or 2", i);
      // (E4M3, likewise carried by the grouped block-scaled GEMM)
      pj_precision plain = x.prec;
      plain.split_terms = 1;
      plain.compute = PJ_BF16;
      PJ_TRY(conv_geom(x.M, x.K, x.N, x.block, x.R, &x.basis, &plain, &cg[i]));
      if (!cg[i].box || x.R % 64)
        return fail(PJ_EUNSUPPORTED, "batch entry %d: batched CONV takes the Haar basis and R a multiple of 64", i);
      if (x.in_dtype != PJ_F32 || x.out_dtype != PJ_F32)
        return fail(PJ_EUNSUPPORTED, "batch entry %d: CONV takes PJ_F32 in and out", i);
      if (!x.A || !x.B || !x.Y) return fail(PJ_EINVAL, "batch entry %d: NULL pointer", i);
    } else {
      return fail(PJ_EINVAL, "batch entry %d: unknown op %d", i, x.op);
    }
  }
  b.basis_off = L.take(kBasisBytes * (b.bases.size() ? b.bases.size() : 1));
  for (int i = 0; i < n; ++i) {
    const pj_batch_desc& x = d[i];
    if (x.op == PJ_OP_GEMM) {
      const GemmGeom& g = gg[i];
      if (g.M == 0 || g.N == 0) continue;
      const int64_t pitch = g.Kp_pad * g.nsplit;
      const int64_t NG = ceil_div(g.K, g.L);
      const size_t ac = L.take(2 * pitch * g.M), bd = L.take(2 * pitch * g.N);
      const int bid = basis_index[std::make_tuple(x.basis.kind, x.basis.L, g.lp1, x.basis.user_C)];
      (void)NG;
      const float* Cs = nullptr;
      const float* Ds = nullptr;
      if (ws) {
        BasisDev area = basis_area(static_cast<char*>(ws) + b.basis_off + kBasisBytes * bid - kHeaderBytes);
        Cs = area.Cs32;
        Ds = area.Ds32;
      }
      // L = 8 operands that TMA can address go to the TMA-staged job launches, and
      // so do the E4M3 sides the projection quantises itself when TMA cannot
      // address them (their rows read by bulk copies, which for BF16 output
      // measured slower than the per-group job kernels); the rest go to the
      // per-group job kernels.
      const float* CsT = nullptr;
      if (ws) {
        BasisDev area = basis_area(static_cast<char*>(ws) + b.basis_off + kBasisBytes * bid - kHeaderBytes);
        CsT = area.CsT32;
      }
      const bool tma_ok = g.L == 8 && g.lp1 >= 1 && g.lp1 <= 8;
      const int tcls = tma_class(x.in_dtype, g.lp1);
      RowsJob r = make_rows_job(x.A, x.lda, x.in_dtype, g, Cs, ptr<uint16_t>(ws, ac));
      ColsJob c = make_cols_job(x.B, x.ldb, x.in_dtype, g, Ds, ptr<uint16_t>(ws, bd));
      const bool a_map = tma_ok && tma_projection_ok(x.A, x.in_dtype, g.K, g.M, x.lda);
      const bool b_map = tma_ok && tma_projection_ok(x.B, x.in_dtype, g.N, g.K, x.ldb);
      // E4M3: the TMA job projection writes E4M3 components and scales itself where it
      // can; the other sides are projected to BF16 hi/lo and quantised
      const bool e4 = g.compute == PJ_E4M3;
      const bool a_q = e4 && project_mx_fusable(g, 0) &&
                       (a_map || (tma_ok && bulk_projection_ok(x.A, x.in_dtype, g.K, g.M, x.lda)));
      const bool b_q = e4 && project_mx_fusable(g, 1) &&
                       (b_map || (tma_ok && bulk_projection_ok(x.B, x.in_dtype, g.N, g.K, x.ldb)));
      const bool a_tma = a_map || a_q, b_tma = b_map || b_q;
      MxQuantSide qa{}, qb{};
      size_t aq = 0, bq = 0, sfq = 0, sfp = 0;
      int bn = 0;
      const int64_t qpitch = g.Kq_pad * g.qsplit;
      if (e4) {
        bn = pick_bn(g.M, 16, kMxTileRows, b.tune);
        aq = L.take(qpitch * g.M);
        bq = L.take(qpitch * g.N);
        sfq = L.take(mx_sf_bytes(g.M, 1, g.Kq_pad, g.qsplit, bn));
        sfp = L.take(mx_sf_bytes(g.N, 0, g.Kq_pad, g.qsplit));
        qa = make_mx_side(r.Ac, g.Kp_pad, g.M, ptr<uint8_t>(ws, aq), g.Kq_pad, g.qsplit, ptr<uint8_t>(ws, sfq), 1, bn);
        qb = make_mx_side(c.Bd, g.Kp_pad, g.N, ptr<uint8_t>(ws, bq), g.Kq_pad, g.qsplit, ptr<uint8_t>(ws, sfp), 0);
      }
      if (a_tma) {
        TmaSpec sp{x.A, x.lda, x.in_dtype, 0, g, CsT, r.Ac};
        if (a_q) {
          sp.quant = 1;
          sp.q = qa;
        }
        sp.bulk = a_map ? 0 : 1;
        const int cl = tcls + (a_q ? 16 : 0) + (a_map ? 0 : 32);
        b.tma[cl].push_back(sp);
        b.tma_units[cl] += tma_job_units(g, 0) * (a_map ? 1 : 2);   // int4 per unit
      } else {
        b.rows[projection_class(r.in_bf16, r.L)].push_back(r);
      }
      if (b_tma) {
        TmaSpec sp{x.B, x.ldb, x.in_dtype, 1, g, Ds, c.Bd};
        if (b_q) {
          sp.quant = 1;
          sp.q = qb;
        }
        sp.bulk = b_map ? 0 : 1;
        const int cl = tcls + (b_q ? 16 : 0) + (b_map ? 0 : 32);
        b.tma[cl].push_back(sp);
        b.tma_units[cl] += tma_job_units(g, 1) * (b_map ? 1 : 2);
      } else {
        b.cols[projection_class(c.in_bf16, c.L)].push_back(c);
      }
      if (e4) {
        // the sides the quantiser pass still handles
        if (!a_q) b.qsides.push_back(qa);
        if (!b_q) b.qsides.push_back(qb);
        MxGemmArgs m{};
        m.Q = ptr<uint8_t>(ws, aq); m.P = ptr<uint8_t>(ws, bq);
        m.sfQ = ptr<uint8_t>(ws, sfq); m.sfP = ptr<uint8_t>(ws, sfp);
        m.rowsQ = g.M; m.rowsP = g.N; m.pitch = qpitch; m.Kq_pad = g.Kq_pad; m.qsplit = g.qsplit;
        m.Y = x.Y; m.ldy = x.ldy; m.out_dtype = x.out_dtype; m.bn = bn;
        const int stages = static_cast<int>(g.Kq_pad / 128) * (g.qsplit == 1 ? 1 : 3);
        b.planned.push_back(GemmPlanned{1, static_cast<int>(b.mx.size()), static_cast<int>(ceil_div(g.M, bn)),
                                        static_cast<int>(ceil_div(g.N, 128)), stages, bn,
                                        split_cap(stages, x.out_dtype == PJ_F32, b.tune), x.out_dtype == PJ_BF16});
        b.mx.push_back(m);
      } else {
        GemmTcArgs a;
        a.Q = r.Ac; a.ldq = pitch; a.rowsQ = g.M;
        a.P = c.Bd; a.ldp = pitch; a.rowsP = g.N;
        a.xdim = pitch; a.kdim = g.Kp_pad;
        a.Y = x.Y; a.ldy = x.ldy; a.out_dtype = x.out_dtype;
        if (g.nsplit == 1) {
          a.nseg = 1;
          a.segQ[0] = a.segP[0] = 0;
        } else {
          a.nseg = 3;
          a.segQ[0] = 0; a.segP[0] = 0;
          a.segQ[1] = 0; a.segP[1] = g.Kp_pad;
          a.segQ[2] = g.Kp_pad; a.segP[2] = 0;
        }
        a.bn = pick_bn(g.M, 32, 256, b.tune);
        const int stages = static_cast<int>(ceil_div(g.Kp_pad, 64)) * a.nseg;
        b.planned.push_back(GemmPlanned{0, static_cast<int>(b.gemms.size()), static_cast<int>(ceil_div(g.M, a.bn)),
                                        static_cast<int>(ceil_div(g.N, 128)), stages, a.bn,
                                        split_cap(stages, x.out_dtype == PJ_F32, b.tune), x.out_dtype == PJ_BF16});
        b.gemms.push_back(a);
      }
    } else {
      const ConvGeom& g = cg[i];
      // E4M3: the BF16 hi + lo of the projected signal and templates feed the quantisers
      const bool e4 = x.prec.compute == PJ_E4M3;
      const int nsplit = e4 ? 2 : x.prec.split_terms;
      const int64_t Kpad = round_up(g.R + 127, 64);
      const int64_t Kq = round_up(Kpad, 128);
      const float scale = 1.0f / sqrtf(static_cast<float>(g.Lb));
      std::vector<uint16_t*> kts(g.nt);
      for (int64_t t = 0; t < g.nt; ++t) {
        const size_t kt = L.take(2 * 128 * Kpad * nsplit);
        TplJob tj{};
        tj.k = static_cast<const float*>(x.B) + t * g.T;
        tj.Kt = ptr<uint16_t>(ws, kt);
        tj.R = g.R; tj.Kpad = Kpad; tj.ldk = Kpad * nsplit; tj.Lb = g.Lb; tj.nsplit = nsplit; tj.scale = scale;
        b.tpl.push_back(tj);
        kts[t] = tj.Kt;
      }
      // E4M3: each template's Toeplitz rows quantised per run of 32 (the quantiser pass)
      std::vector<uint8_t*> pqs(g.nt), sfps(g.nt);
      if (e4)
        for (int64_t t = 0; t < g.nt; ++t) {
          const size_t pq = L.take(128 * Kq), sfp = L.take(mx_sf_bytes(128, 0, Kq, 1));
          pqs[t] = ptr<uint8_t>(ws, pq);
          sfps[t] = ptr<uint8_t>(ws, sfp);
          b.qsides.push_back(make_mx_side(kts[t], Kpad, 128, pqs[t], Kq, 1, sfps[t], 0));
        }
      for (int phi = 0; phi < g.Lb; ++phi) {
        const int64_t lags_phi = g.lags > phi ? ceil_div(g.lags - phi, g.Lb) : 0;
        if (lags_phi == 0) continue;
        const int64_t rows_alloc = ceil_div(lags_phi + g.R - 1, 128) + 1;
        const size_t q = L.take(2 * 128 * rows_alloc * nsplit);
        SigJob sj{};
        sj.s = static_cast<const float*>(x.A); sj.Q = ptr<uint16_t>(ws, q);
        sj.Qlo = nsplit > 1 ? ptr<uint16_t>(ws, q + 2 * 128 * rows_alloc) : nullptr;
        sj.S = g.S; sj.n = rows_alloc * 128; sj.Lb = g.Lb; sj.phi = phi; sj.scale = scale;
        b.sig.push_back(sj);
        if (e4) {
          const int64_t rowsQ = ceil_div(lags_phi, 128);
          const int bn = pick_bn(rowsQ, 16, kMxTileRows, b.tune);
          const int kc = static_cast<int>(Kq / 128);
          const int64_t tiles_m = ceil_div(rowsQ, bn);
          const size_t qe = L.take(128 * rows_alloc), bsc = L.take(4 * rows_alloc);
          const size_t sfq = L.take(static_cast<size_t>(tiles_m * kc * 1024));
          b.sigq.push_back(SigQJob{sj.Q, sj.Qlo, ptr<uint8_t>(ws, qe), ptr<uint8_t>(ws, bsc), 4 * rows_alloc, 0});
          b.sfx.push_back(SfExpJob{ptr<uint8_t>(ws, bsc), ptr<uint8_t>(ws, sfq), rows_alloc,
                                   tiles_m * kc * bn * 4, 0, kc, bn});
          for (int64_t t = 0; t < g.nt; ++t) {
            MxGemmArgs m{};
            m.Q = ptr<uint8_t>(ws, qe); m.q_pitch = 128; m.q_rows = rows_alloc; m.rowsQ = rowsQ;
            m.P = pqs[t]; m.pitch = Kq; m.rowsP = 128;
            m.sfQ = ptr<uint8_t>(ws, sfq); m.sfP = sfps[t];
            m.Kq_pad = Kq; m.qsplit = 1;
            m.Y = static_cast<float*>(x.Y) + phi * g.nt + t;
            m.ldy = 128; m.out_dtype = PJ_F32; m.bn = bn;
            m.conv_mode = 1;
            m.conv_stride = static_cast<int64_t>(g.Lb) * g.nt;
            m.conv_limit = lags_phi;
            b.planned.push_back(GemmPlanned{1, static_cast<int>(b.mx.size()), static_cast<int>(tiles_m), 1, kc, bn,
                                            1, false});
            b.mx.push_back(m);
          }
          continue;
        }
        for (int64_t t = 0; t < g.nt; ++t) {
          GemmTcArgs a;
          a.Q = sj.Q; a.ldq = 128; a.rowsQ = ceil_div(lags_phi, 128);
          a.P = kts[t]; a.ldp = Kpad * nsplit; a.rowsP = 128;
          a.xdim = Kpad * nsplit; a.kdim = Kpad;
          if (nsplit == 1) {
            a.nseg = 1;
            a.segQ[0] = a.segP[0] = 0;
          } else {
            // hi.hi + hi.lo + lo.hi; in the row-split view segQ is a row offset
            a.nseg = 3;
            a.segQ[0] = 0;         a.segP[0] = 0;
            a.segQ[1] = 0;         a.segP[1] = Kpad;
            a.segQ[2] = rows_alloc; a.segP[2] = 0;
          }
          a.Y = static_cast<float*>(x.Y) + phi * g.nt + t;
          a.ldy = 128; a.out_dtype = PJ_F32;
          a.conv_mode = 1; a.q_rows_alloc = rows_alloc * nsplit;
          a.conv_stride = static_cast<int64_t>(g.Lb) * g.nt;
          a.conv_limit = lags_phi;
          a.bn = 256;
          const int stages = static_cast<int>(ceil_div(Kpad, 64)) * a.nseg;
          b.planned.push_back(GemmPlanned{0, static_cast<int>(b.gemms.size()),
                                          static_cast<int>(ceil_div(a.rowsQ, 256)), 1, stages, 256, 1, false});
          b.gemms.push_back(a);
        }
      }
    }
  }
  // job tables, instance table and tile list
  int64_t blk = 0;
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    blk = 0;
    for (auto& r : b.rows[cls]) { r.block0 = blk; blk += rows_job_blocks(r); }
    b.rows_total[cls] = blk;
    blk = 0;
    for (auto& c : b.cols[cls]) { c.block0 = blk; blk += cols_job_blocks(c); }
    b.cols_total[cls] = blk;
  }
  blk = 0;
  for (auto& s : b.sig) { s.block0 = blk; blk += ceil_div(s.n, 256); }
  b.sig_total = blk;
  blk = 0;
  for (auto& t : b.tpl) { t.block0 = blk; blk += ceil_div(128 * t.Kpad, 256); }
  b.tpl_total = blk;
  blk = 0;
  for (auto& q : b.sigq) { q.block0 = blk; blk += ceil_div(q.nblk, 256); }
  b.sigq_total = blk;
  blk = 0;
  for (auto& f : b.sfx) { f.block0 = blk; blk += ceil_div(f.total, 256); }
  b.sfx_total = blk;
  b.sigq_map_off = L.take(sizeof(int) * (b.sigq_total + 1));
  b.sfx_map_off = L.take(sizeof(int) * (b.sfx_total + 1));
  b.sigq_off = L.take(sizeof(SigQJob) * (b.sigq.size() + 1));
  b.sfx_off = L.take(sizeof(SfExpJob) * (b.sfx.size() + 1));
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    b.rows_map_off[cls] = L.take(sizeof(int) * (b.rows_total[cls] + 1));
    b.cols_map_off[cls] = L.take(sizeof(int) * (b.cols_total[cls] + 1));
  }
  b.sig_map_off = L.take(sizeof(int) * (b.sig_total + 1));
  b.tpl_map_off = L.take(sizeof(int) * (b.tpl_total + 1));
  for (int tc = 0; tc < kTmaClasses; ++tc) {
    b.tma_jobs_off[tc] = L.take(sizeof(TmaJob) * (b.tma[tc].size() + 1));
    b.tma_units_off[tc] = L.take(sizeof(int4) * (b.tma_units[tc] + 1));
  }
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    b.rows_off[cls] = L.take(sizeof(RowsJob) * (b.rows[cls].size() + 1));
    b.cols_off[cls] = L.take(sizeof(ColsJob) * (b.cols[cls].size() + 1));
  }
  b.sig_off = L.take(sizeof(SigJob) * (b.sig.size() + 1));
  b.tpl_off = L.take(sizeof(TplJob) * (b.tpl.size() + 1));
  // quantiser sides and zero jobs (blocks laid out job by job)
  blk = 0;
  for (auto& q : b.qsides) { q.block0 = blk; blk += mx_side_blocks(q); }
  b.qsides_total = blk;
  for (const auto& pl : b.planned)
    if (pl.cap > 1) {
      const int64_t M = pl.kind ? b.mx[pl.index].rowsQ : b.gemms[pl.index].rowsQ;
      const int64_t N = pl.kind ? b.mx[pl.index].rowsP : b.gemms[pl.index].rowsP;
      const int64_t ld = pl.kind ? b.mx[pl.index].ldy : b.gemms[pl.index].ldy;
      void* Y = pl.kind ? b.mx[pl.index].Y : b.gemms[pl.index].Y;
      b.zeros.push_back(ZeroJob{static_cast<float*>(Y), M, N, ld, 0});
    }
  blk = 0;
  for (auto& z : b.zeros) { z.block0 = blk; blk += ceil_div(z.rows, 4); }
  b.zero_total = blk;
  b.qsides_off = L.take(sizeof(MxQuantSide) * (b.qsides.size() + 1));
  b.qsides_map_off = L.take(sizeof(int) * (b.qsides_total + 1));
  b.zero_off = L.take(sizeof(ZeroJob) * (b.zeros.size() + 1));
  b.zero_map_off = L.take(sizeof(int) * (b.zero_total + 1));
  b.insts_off = L.take(sizeof(GemmInst) * (b.gemms.size() + 1));
  b.mx_off = L.take(sizeof(MxInst) * (b.mx.size() + 1));
  // tile lists sized for the largest split the tuner may choose
  int tiles = 0, mx_tiles = 0;
  // (plus, for paired BF16 tiles, at most one stand-in tile per piece of an instance)
  for (const auto& pl : b.planned) (pl.kind ? mx_tiles : tiles) += pl.tiles_m * pl.tiles_n * pl.cap + (pl.kind ? 0 : pl.cap);
  b.tiles_cap = tiles;
  b.mx_tiles_cap = mx_tiles;
  b.tiles_off = L.take(sizeof(GemmTile) * (tiles + 1));
  b.mx_tiles_off = L.take(sizeof(GemmTile) * (mx_tiles + 1));
  b.cta_off_off = L.take(sizeof(int) * (kMaxCtas + 1));
  b.mx_cta_off = L.take(sizeof(int) * (kMaxCtas + 1));
  b.total = L.off;
  return PJ_OK;
}

// ------------------------------------------------------------ the tuner --

double tile_cost(const Tuning& t, int stages, int bn, bool out_bf16, bool red) {
  const double out_kb = bn * 128.0 * (out_bf16 ? 2 : 4) / 1024.0 * (red ? 2.0 : 1.0);
  return t.t_tile + stages * t.t_stage * (bn < 64 ? 64 : bn) / 256.0 + out_kb * t.t_out_kb;
}

struct Schedule {
  std::vector<GemmTile> tiles;  // CTA by CTA
  std::vector<int> cta_off;     // ctas + 1 entries
  double makespan = 0, total = 0;
  int splits = 0;
  bool paired = false;          // CTAs 2c and 2c + 1 form a cluster (see schedule_kind)
};

// Tiles of the instances of one kernel (kind), with the splits chosen, dealt to
// the CTAs (paired: to clusters of two CTAs, see Item).
Schedule schedule_kind(const Built& b, int kind, int sms, bool paired) {
  const Tuning& t = b.tune;
  std::vector<const GemmPlanned*> ins;
  for (const auto& pl : b.planned)
    if (pl.kind == kind) ins.push_back(&pl);
  std::vector<int> split(ins.size(), 1);
  int64_t ntiles = 0;
  double total = 0;
  for (const auto* pl : ins) {
    ntiles += static_cast<int64_t>(pl->tiles_m) * pl->tiles_n;
    total += pl->tiles_m * pl->tiles_n * tile_cost(t, pl->stages, pl->bn, pl->out_bf16, false);
  }
  Schedule S;
  if (ntiles == 0) {
    S.cta_off.assign(1, 0);
    return S;
  }
  // Split the reduced dimension of instances whose tiles are long next to the
  // average load of a CTA (so that no single tile sets the makespan).
  if (t.schedule != 1) {
    for (int pass = 0; pass < 4; ++pass) {
      const int64_t ctas = ntiles < sms ? ntiles : sms;
      const double ideal = total / static_cast<double>(ctas);
      bool changed = false;
      for (size_t i = 0; i < ins.size(); ++i) {
        const GemmPlanned& pl = *ins[i];
        while (split[i] < pl.cap &&
               tile_cost(t, pl.stages / split[i], pl.bn, pl.out_bf16, split[i] > 1) > 0.5 * ideal) {
          const double before = pl.tiles_m * pl.tiles_n * split[i] *
                                tile_cost(t, pl.stages / split[i], pl.bn, pl.out_bf16, split[i] > 1);
          split[i] *= 2;
          total += pl.tiles_m * pl.tiles_n * split[i] *
                       tile_cost(t, pl.stages / split[i], pl.bn, pl.out_bf16, true) - before;
          ntiles += static_cast<int64_t>(pl.tiles_m) * pl.tiles_n * (split[i] / 2);
          changed = true;
        }
      }
      if (!changed) break;
    }
  }
  // An item is the work of one CTA or, paired, of the two CTAs of a cluster:
  // t[0] for the CTA of rank 0, t[1] for rank 1.  Paired tiles are neighbouring
  // tile columns of one tile row (they share that row's A_c tiles); the last
  // column of an odd number of columns pairs with the same column of the next
  // tile row, each CTA loading its own A_c tile (flag 1), and a last one left
  // over pairs with a stand-in copy of itself whose output is not written
  // (flags 1 | 2).  Both tiles of an item have the same K stages.
  struct Item {
    GemmTile t[2];
    double cost;
  };
  std::vector<Item> items;
  items.reserve(static_cast<size_t>(ntiles));
  for (size_t i = 0; i < ins.size(); ++i) {
    const GemmPlanned& pl = *ins[i];
    const int sp = split[i];
    if (sp > 1) ++S.splits;
    for (int k = 0; k < sp; ++k) {
      const int k0 = static_cast<int>(static_cast<int64_t>(pl.stages) * k / sp);
      const int k1 = static_cast<int>(static_cast<int64_t>(pl.stages) * (k + 1) / sp);
      const double cost = tile_cost(t, k1 - k0, pl.bn, pl.out_bf16, sp > 1);
      auto tile = [&](int ti, int tj, int flags) {
        return GemmTile{pl.index, ti, tj, k0, k1, sp > 1 ? 1 : 0, flags, 0};
      };
      if (!paired) {
        for (int ti = 0; ti < pl.tiles_m; ++ti)
          for (int tj = 0; tj < pl.tiles_n; ++tj) items.push_back(Item{{tile(ti, tj, 0), tile(ti, tj, 0)}, cost});
        continue;
      }
      for (int ti = 0; ti < pl.tiles_m; ++ti)
        for (int tj = 0; tj + 1 < pl.tiles_n; tj += 2) items.push_back(Item{{tile(ti, tj, 0), tile(ti, tj + 1, 0)}, cost});
      if (pl.tiles_n % 2) {
        const int tj = pl.tiles_n - 1;
        for (int ti = 0; ti + 1 < pl.tiles_m; ti += 2) items.push_back(Item{{tile(ti, tj, 1), tile(ti + 1, tj, 1)}, cost});
        if (pl.tiles_m % 2) items.push_back(Item{{tile(pl.tiles_m - 1, tj, 1), tile(pl.tiles_m - 1, tj, 3)}, cost});
      }
    }
  }
  // units that take items: CTAs, or clusters of two when paired
  const int slots = paired ? sms / 2 : sms;
  const int units = static_cast<int>(items.size() < static_cast<size_t>(slots) ? items.size() : slots);
  std::vector<std::vector<int>> per(units);
  std::vector<double> load(units, 0.0);
  if (t.schedule != 2) {
    // longest reduced K first (measured faster than costliest first), dealt
    // round-robin, so the tiles of one instance run side by side and share
    // their operand panels in L2
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = static_cast<int>(k);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
      return items[a].t[0].k1 - items[a].t[0].k0 > items[c].t[0].k1 - items[c].t[0].k0;
    });
    for (size_t k = 0; k < order.size(); ++k) {
      per[k % units].push_back(order[k]);
      load[k % units] += items[order[k]].cost;
    }
  } else {
    // LPT: costliest item first onto the least-loaded unit
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = static_cast<int>(k);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return items[a].cost > items[c].cost; });
    std::vector<std::pair<double, int>> heap;
    for (int c = 0; c < units; ++c) heap.push_back({0.0, c});
    auto cmp = [](const std::pair<double, int>& a, const std::pair<double, int>& c) {
      return a.first > c.first || (a.first == c.first && a.second > c.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (int k : order) {
      std::pop_heap(heap.begin(), heap.end(), cmp);
      auto& top = heap.back();
      per[top.second].push_back(k);
      top.first += items[k].cost;
      load[top.second] = top.first;
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
  S.cta_off.push_back(0);
  for (int c = 0; c < units; ++c) {
    for (int r = 0; r < (paired ? 2 : 1); ++r) {
      for (int k : per[c]) S.tiles.push_back(items[k].t[r]);
      S.cta_off.push_back(static_cast<int>(S.tiles.size()));
      S.total += load[c];
    }
    S.makespan = load[c] > S.makespan ? load[c] : S.makespan;
  }
  S.paired = paired;
  return S;
}

// block -> job index for jobs laid out by block0 (the last job runs to `total`).
template <typename Job>
std::vector<int> job_map(const std::vector<Job>& jobs, int64_t total) {
  std::vector<int> m(static_cast<size_t>(total));
  for (size_t j = 0; j < jobs.size(); ++j) {
    const int64_t end = j + 1 < jobs.size() ? jobs[j + 1].block0 : total;
    for (int64_t b = jobs[j].block0; b < end; ++b) m[static_cast<size_t>(b)] = static_cast<int>(j);
  }
  return m;
}

template <typename T>
pj_status upload(const std::vector<T>& v, void* ws, size_t off, cudaStream_t st) {
  if (!v.empty())
    PJ_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(ws) + off, v.data(), sizeof(T) * v.size(),
                                cudaMemcpyHostToDevice, st));
  return PJ_OK;
}

}  // namespace

extern "C" {

size_t proj_batch_workspace_size_tuned(const pj_batch_desc* descs, int32_t n, const pj_batch_tuning* tuning) {
  Built b;
  if (layout(descs, n, tuning, nullptr, &b) != PJ_OK) return 0;
  return b.total;
}

size_t proj_batch_workspace_size(const pj_batch_desc* descs, int32_t n) {
  return proj_batch_workspace_size_tuned(descs, n, nullptr);
}

pj_status proj_batch_plan_create(const pj_batch_desc* descs, int32_t n, void* workspace, size_t ws_bytes,
                                 void* stream, pj_batch_plan** plan) {
  return proj_batch_plan_create_tuned(descs, n, nullptr, workspace, ws_bytes, stream, plan);
}

pj_status proj_batch_plan_create_tuned(const pj_batch_desc* descs, int32_t n, const pj_batch_tuning* tuning,
                                       void* workspace, size_t ws_bytes, void* stream, pj_batch_plan** plan) {
  if (!plan) return fail(PJ_EINVAL, "plan is NULL");
  *plan = nullptr;
  Built b;
  PJ_TRY(layout(descs, n, tuning, nullptr, &b));
  if (!workspace) return fail(PJ_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(PJ_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < b.total) return fail(PJ_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, b.total);
  Built w;
  PJ_TRY(layout(descs, n, tuning, workspace, &w));
  int sms = 0;
  PJ_TRY(device_sms(&sms));
  if (sms > kMaxCtas) sms = kMaxCtas;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PJ_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(int), st));
  // projection bases (FP64 on the GPU, once per plan)
  for (size_t id = 0; id < w.bases.size(); ++id) {
    const auto& key = w.bases[id];
    BasisDev area = basis_area(static_cast<char*>(workspace) + w.basis_off + kBasisBytes * id - kHeaderBytes);
    const int kind = std::get<0>(key), L = std::get<1>(key), lp1 = std::get<2>(key);
    if (kind == PJ_BASIS_USER)
      PJ_CUDA_TRY(cudaMemcpyAsync(area.U64, std::get<3>(key), sizeof(double) * L * L, cudaMemcpyHostToDevice, st));
    PJ_CUDA_TRY(launch_basis_build(kind, L, lp1, area, error_word(workspace), st));
  }
  // instance tables and the tuned schedules of the two grouped launches
  // BF16 products on CTA pairs unless the tuning asks for solo CTAs
  const bool paired = PJ_CTA_PAIRS && !w.tune.solo && sms >= 2;
  std::vector<GemmInst> insts(w.gemms.size());
  for (size_t i = 0; i < w.gemms.size(); ++i) {
    w.gemms[i].pair = paired ? 1 : 0;
    if (!build_gemm_inst(w.gemms[i], &insts[i])) return fail(PJ_EINVAL, "could not encode tensor maps for batch entry");
  }
  std::vector<MxInst> mxi(w.mx.size());
  for (size_t i = 0; i < w.mx.size(); ++i)
    if (!build_mx_inst(w.mx[i], &mxi[i])) return fail(PJ_EINVAL, "could not encode tensor maps for batch entry");
  const Schedule S0 = schedule_kind(w, 0, sms, paired);
  const Schedule S1 = schedule_kind(w, 1, sms, false);
  if (S0.tiles.size() > static_cast<size_t>(w.tiles_cap) || S1.tiles.size() > static_cast<size_t>(w.mx_tiles_cap))
    return fail(PJ_EINVAL, "internal: schedule exceeds its reserved tile list");
  // zero jobs are needed only for the instances the schedules actually split
  std::vector<ZeroJob> zeros;
  {
    std::vector<char> split0(w.gemms.size(), 0), split1(w.mx.size(), 0);
    for (const auto& t : S0.tiles) if (t.red) split0[t.inst] = 1;
    for (const auto& t : S1.tiles) if (t.red) split1[t.inst] = 1;
    int64_t blk = 0;
    for (const auto& pl : w.planned) {
      if (!(pl.kind ? split1[pl.index] : split0[pl.index])) continue;
      ZeroJob z{};
      if (pl.kind) {
        z.Y = static_cast<float*>(w.mx[pl.index].Y); z.rows = w.mx[pl.index].rowsQ;
        z.cols = w.mx[pl.index].rowsP; z.ld = w.mx[pl.index].ldy;
      } else {
        z.Y = static_cast<float*>(w.gemms[pl.index].Y); z.rows = w.gemms[pl.index].rowsQ;
        z.cols = w.gemms[pl.index].rowsP; z.ld = w.gemms[pl.index].ldy;
      }
      z.block0 = blk;
      blk += ceil_div(z.rows, 4);
      zeros.push_back(z);
    }
  }
  int64_t zero_blocks = 0;
  for (const auto& z : zeros) zero_blocks = z.block0 + ceil_div(z.rows, 4);
  if (zeros.size() > w.zeros.size() || zero_blocks > w.zero_total)
    return fail(PJ_EINVAL, "internal: zero jobs exceed their reserved table");
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    PJ_TRY(upload(w.rows[cls], workspace, w.rows_off[cls], st));
    PJ_TRY(upload(w.cols[cls], workspace, w.cols_off[cls], st));
  }
  PJ_TRY(upload(w.sig, workspace, w.sig_off, st));
  PJ_TRY(upload(w.tpl, workspace, w.tpl_off, st));
  PJ_TRY(upload(w.sigq, workspace, w.sigq_off, st));
  PJ_TRY(upload(w.sfx, workspace, w.sfx_off, st));
  // TMA jobs (tensor maps encoded now) and their unit lists, job by job
  std::vector<std::vector<TmaJob>> tma_jobs(kTmaClasses);
  std::vector<std::vector<int4>> tma_units(kTmaClasses);
  for (int tc = 0; tc < kTmaClasses; ++tc) {
    for (size_t j = 0; j < w.tma[tc].size(); ++j) {
      const TmaSpec& sp = w.tma[tc][j];
      TmaJob J;
      if (!make_tma_job(sp.X, sp.ld, sp.in_dtype, sp.cols, sp.g, sp.coef, sp.out, &J, sp.quant ? &sp.q : nullptr,
                        sp.bulk != 0))
        return fail(PJ_EINVAL, "could not encode a projection tensor map for a batch entry");
      tma_jobs[tc].push_back(J);
      if (sp.bulk) {
        bulk_job_units(J, sp.in_dtype, static_cast<int>(j), tma_units[tc]);
      } else {
        for (int uy = 0; uy < J.units_y; ++uy)
          for (int ux = 0; ux < J.units_x; ++ux) tma_units[tc].push_back(make_int4(static_cast<int>(j), ux, uy, 0));
      }
    }
    PJ_TRY(upload(tma_jobs[tc], workspace, w.tma_jobs_off[tc], st));
    PJ_TRY(upload(tma_units[tc], workspace, w.tma_units_off[tc], st));
  }
  // the maps must outlive the asynchronous copies: they are uploaded before the synchronize below
  std::vector<std::vector<int>> maps;
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    maps.push_back(job_map(w.rows[cls], w.rows_total[cls]));
    PJ_TRY(upload(maps.back(), workspace, w.rows_map_off[cls], st));
    maps.push_back(job_map(w.cols[cls], w.cols_total[cls]));
    PJ_TRY(upload(maps.back(), workspace, w.cols_map_off[cls], st));
  }
  maps.push_back(job_map(w.sig, w.sig_total));
  PJ_TRY(upload(maps.back(), workspace, w.sig_map_off, st));
  maps.push_back(job_map(w.tpl, w.tpl_total));
  PJ_TRY(upload(maps.back(), workspace, w.tpl_map_off, st));
  maps.push_back(job_map(w.sigq, w.sigq_total));
  PJ_TRY(upload(maps.back(), workspace, w.sigq_map_off, st));
  maps.push_back(job_map(w.sfx, w.sfx_total));
  PJ_TRY(upload(maps.back(), workspace, w.sfx_map_off, st));
  maps.push_back(job_map(w.qsides, w.qsides_total));
  PJ_TRY(upload(maps.back(), workspace, w.qsides_map_off, st));
  maps.push_back(job_map(zeros, zero_blocks));
  PJ_TRY(upload(maps.back(), workspace, w.zero_map_off, st));
  PJ_TRY(upload(w.qsides, workspace, w.qsides_off, st));
  PJ_TRY(upload(zeros, workspace, w.zero_off, st));
  PJ_TRY(upload(insts, workspace, w.insts_off, st));
  PJ_TRY(upload(mxi, workspace, w.mx_off, st));
  PJ_TRY(upload(S0.tiles, workspace, w.tiles_off, st));
  PJ_TRY(upload(S1.tiles, workspace, w.mx_tiles_off, st));
  PJ_TRY(upload(S0.cta_off, workspace, w.cta_off_off, st));
  PJ_TRY(upload(S1.cta_off, workspace, w.mx_cta_off, st));
  PJ_CUDA_TRY(cudaStreamSynchronize(st));
  int code = 0;
  PJ_CUDA_TRY(cudaMemcpy(&code, workspace, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) return fail(PJ_EINVAL, "a batch basis was rejected on the device (singular user matrix)");
  pj_batch_plan* p = new pj_batch_plan;
  p->ws = workspace;
  p->ws_bytes = ws_bytes;
  for (int tc = 0; tc < kTmaClasses; ++tc) {
    p->d_tma_jobs[tc] = ptr<TmaJob>(workspace, w.tma_jobs_off[tc]);
    p->d_tma_units[tc] = ptr<int4>(workspace, w.tma_units_off[tc]);
    p->tma_units[tc] = static_cast<int64_t>(tma_units[tc].size()) / (tc >= 32 ? 2 : 1);   // bulk units: two int4
  }
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    p->d_rows[cls] = ptr<RowsJob>(workspace, w.rows_off[cls]);
    p->d_cols[cls] = ptr<ColsJob>(workspace, w.cols_off[cls]);
    p->n_rows[cls] = static_cast<int>(w.rows[cls].size());
    p->n_cols[cls] = static_cast<int>(w.cols[cls].size());
    p->rows_of[cls] = ptr<int>(workspace, w.rows_map_off[cls]);
    p->cols_of[cls] = ptr<int>(workspace, w.cols_map_off[cls]);
    for (const auto& r : w.rows[cls]) p->rows_blocks[cls] = r.block0 + rows_job_blocks(r);
    for (const auto& c : w.cols[cls]) p->cols_blocks[cls] = c.block0 + cols_job_blocks(c);
  }
  p->d_sig = ptr<SigJob>(workspace, w.sig_off);
  p->d_tpl = ptr<TplJob>(workspace, w.tpl_off);
  p->n_sig = static_cast<int>(w.sig.size());
  p->n_tpl = static_cast<int>(w.tpl.size());
  p->sig_of = ptr<int>(workspace, w.sig_map_off);
  p->tpl_of = ptr<int>(workspace, w.tpl_map_off);
  for (const auto& s : w.sig) p->sig_blocks = s.block0 + ceil_div(s.n, 256);
  for (const auto& t : w.tpl) p->tpl_blocks = t.block0 + ceil_div(128 * t.Kpad, 256);
  p->d_sigq = ptr<SigQJob>(workspace, w.sigq_off);
  p->d_sfx = ptr<SfExpJob>(workspace, w.sfx_off);
  p->sigq_of = ptr<int>(workspace, w.sigq_map_off);
  p->sfx_of = ptr<int>(workspace, w.sfx_map_off);
  p->sigq_blocks = w.sigq_total;
  p->sfx_blocks = w.sfx_total;
  p->d_insts = ptr<GemmInst>(workspace, w.insts_off);
  p->d_tiles = ptr<GemmTile>(workspace, w.tiles_off);
  p->d_cta_off = ptr<int>(workspace, w.cta_off_off);
  p->ctas = static_cast<int>(S0.cta_off.size()) - 1;
  p->paired = S0.paired ? 1 : 0;
  p->d_mx = ptr<MxInst>(workspace, w.mx_off);
  p->d_mx_tiles = ptr<GemmTile>(workspace, w.mx_tiles_off);
  p->d_mx_cta_off = ptr<int>(workspace, w.mx_cta_off);
  p->mx_ctas = static_cast<int>(S1.cta_off.size()) - 1;
  p->d_qsides = ptr<MxQuantSide>(workspace, w.qsides_off);
  p->qsides_of = ptr<int>(workspace, w.qsides_map_off);
  p->qsides_blocks = w.qsides_total;
  p->d_zero = ptr<ZeroJob>(workspace, w.zero_off);
  p->zero_of = ptr<int>(workspace, w.zero_map_off);
  p->zero_blocks = zero_blocks;
  p->sms = sms;
  p->info.gemm_tiles = static_cast<int32_t>(S0.tiles.size());
  p->info.mx_tiles = static_cast<int32_t>(S1.tiles.size());
  p->info.ctas = p->ctas > p->mx_ctas ? p->ctas : p->mx_ctas;
  p->info.split_instances = S0.splits + S1.splits;
  p->info.model_makespan_us = S0.makespan + S1.makespan;
  p->info.model_total_us = S0.total + S1.total;
  *plan = p;
  return PJ_OK;
}

pj_status proj_batch_plan_info(const pj_batch_plan* plan, pj_batch_info* info) {
  if (!plan || !info) return fail(PJ_EINVAL, "plan and info must be non-NULL");
  *info = plan->info;
  return PJ_OK;
}

pj_status proj_batch_run(const pj_batch_plan* plan, void* stream) {
  if (!plan) return fail(PJ_EINVAL, "plan is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PJ_CUDA_TRY(cudaMemsetAsync(plan->ws, 0, sizeof(int), st));
  for (int tc = 0; tc < kTmaClasses; ++tc)
    PJ_CUDA_TRY(launch_project_tma_jobs(tc % 16 >= 8, tc % 8 + 1, plan->d_tma_jobs[tc], plan->d_tma_units[tc],
                                        plan->tma_units[tc], static_cast<int*>(plan->ws), plan->sms, st,
                                        tc % 32 >= 16, tc >= 32));
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    PJ_CUDA_TRY(launch_project_rows_jobs(cls, plan->d_rows[cls], plan->rows_of[cls], plan->rows_blocks[cls], st));
    PJ_CUDA_TRY(launch_project_cols_jobs(cls, plan->d_cols[cls], plan->cols_of[cls], plan->cols_blocks[cls], st));
  }
  if (plan->sig_blocks > 0) {
    batch_signal_kernel<<<static_cast<unsigned>(plan->sig_blocks), 256, 0, st>>>(plan->d_sig, plan->sig_of);
    PJ_CUDA_TRY(cudaGetLastError());
  }
  if (plan->tpl_blocks > 0) {
    batch_toeplitz_kernel<<<static_cast<unsigned>(plan->tpl_blocks), 256, 0, st>>>(plan->d_tpl, plan->tpl_of);
    PJ_CUDA_TRY(cudaGetLastError());
  }
  if (plan->sigq_blocks > 0) {   // after the signal kernel: its hi + lo sequences
    batch_sigquant_kernel<<<static_cast<unsigned>(plan->sigq_blocks), 256, 0, st>>>(plan->d_sigq, plan->sigq_of);
    PJ_CUDA_TRY(cudaGetLastError());
  }
  if (plan->sfx_blocks > 0) {    // after the block scales
    batch_sfexpand_kernel<<<static_cast<unsigned>(plan->sfx_blocks), 256, 0, st>>>(plan->d_sfx, plan->sfx_of);
    PJ_CUDA_TRY(cudaGetLastError());
  }
  if (plan->qsides_blocks > 0)
    PJ_CUDA_TRY(launch_quantize_mx_jobs(plan->d_qsides, plan->qsides_of, plan->qsides_blocks, st));
  if (plan->zero_blocks > 0) {
    batch_zero_kernel<<<static_cast<unsigned>(plan->zero_blocks), 256, 0, st>>>(plan->d_zero, plan->zero_of);
    PJ_CUDA_TRY(cudaGetLastError());
  }
  PJ_CUDA_TRY(launch_gemm_tc_grouped(plan->d_insts, plan->d_tiles, plan->d_cta_off, plan->ctas, plan->paired,
                                     error_word(plan->ws), st));
  PJ_CUDA_TRY(launch_gemm_mx_grouped(plan->d_mx, plan->d_mx_tiles, plan->d_mx_cta_off, plan->mx_ctas,
                                     error_word(plan->ws), st));
  return PJ_OK;
}

void proj_batch_destroy(pj_batch_plan* plan) { delete plan; }

}  // extern "C"
