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
// Tiles are ordered longest first (largest reduced K first), a static LPT
// schedule over the persistent CTAs.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "common.hpp"
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
  GemmInst* d_insts = nullptr;
  GemmTile* d_tiles = nullptr;
  int num_tiles = 0;
  int sms = 0;
};

namespace {

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
  GemmGeom g;
  const float* coef;
  uint16_t* out;
};
inline int tma_class(int in_dtype, int lp1) { return (in_dtype == PJ_BF16 ? 8 : 0) + lp1 - 1; }

struct Built {
  std::vector<TmaSpec> tma[kTmaClasses];
  int64_t tma_units[kTmaClasses] = {};
  size_t tma_jobs_off[kTmaClasses] = {}, tma_units_off[kTmaClasses] = {};
  std::vector<RowsJob> rows[kProjectionClasses];
  std::vector<ColsJob> cols[kProjectionClasses];
  std::vector<SigJob> sig;
  std::vector<TplJob> tpl;
  std::vector<GemmTcArgs> gemms;
  std::vector<std::tuple<int, int, int, const double*>> bases;  // kind, L, lp1, user matrix
  size_t basis_off = 0, rows_off[kProjectionClasses] = {}, cols_off[kProjectionClasses] = {};
  size_t sig_off = 0, tpl_off = 0, insts_off = 0, tiles_off = 0;
  size_t rows_map_off[kProjectionClasses] = {}, cols_map_off[kProjectionClasses] = {}, sig_map_off = 0,
         tpl_map_off = 0;
  int64_t rows_total[kProjectionClasses] = {}, cols_total[kProjectionClasses] = {}, sig_total = 0, tpl_total = 0;
  size_t total = 0;
  int num_tiles = 0;
};

template <typename T>
T* ptr(void* ws, size_t off) {
  return ws ? reinterpret_cast<T*>(static_cast<char*>(ws) + off) : nullptr;
}

// Walks the descriptors, validates them and lays out the workspace.  With
// ws == nullptr only the sizes are computed.
pj_status layout(const pj_batch_desc* d, int n, void* ws, Built* out) {
  if (!d || n < 1) return fail(PJ_EINVAL, "batch needs at least one descriptor");
  Built& b = *out;
  Layout L;
  L.take(kHeaderBytes);
  // distinct GEMM bases, each with its own basis area
  std::map<std::tuple<int, int, int, const double*>, int> basis_index;
  std::vector<GemmGeom> gg(n);
  std::vector<ConvGeom> cg(n);
  for (int i = 0; i < n; ++i) {
    const pj_batch_desc& x = d[i];
    if (x.prec.compute != PJ_BF16) return fail(PJ_EUNSUPPORTED, "batch entry %d: PJ_BF16 compute only", i);
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
      pj_precision plain = x.prec;
      plain.split_terms = 1;
      PJ_TRY(conv_geom(x.M, x.K, x.N, x.block, x.R, &x.basis, &plain, &cg[i]));
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
      // L = 8 operands that TMA can read go to the TMA-staged job launches, the
      // rest to the per-group job kernels.
      const float* CsT = nullptr;
      if (ws) {
        BasisDev area = basis_area(static_cast<char*>(ws) + b.basis_off + kBasisBytes * bid - kHeaderBytes);
        CsT = area.CsT32;
      }
      const bool tma_ok = g.L == 8 && g.lp1 >= 1 && g.lp1 <= 8;
      const int tcls = tma_class(x.in_dtype, g.lp1);
      RowsJob r = make_rows_job(x.A, x.lda, x.in_dtype, g, Cs, ptr<uint16_t>(ws, ac));
      if (tma_ok && tma_projection_ok(x.A, x.in_dtype, g.K, g.M, x.lda)) {
        b.tma[tcls].push_back(TmaSpec{x.A, x.lda, x.in_dtype, 0, g, CsT, r.Ac});
        b.tma_units[tcls] += tma_job_units(g, 0);
      } else {
        b.rows[projection_class(r.in_bf16, r.L)].push_back(r);
      }
      ColsJob c = make_cols_job(x.B, x.ldb, x.in_dtype, g, Ds, ptr<uint16_t>(ws, bd));
      if (tma_ok && tma_projection_ok(x.B, x.in_dtype, g.N, g.K, x.ldb)) {
        b.tma[tcls].push_back(TmaSpec{x.B, x.ldb, x.in_dtype, 1, g, Ds, c.Bd});
        b.tma_units[tcls] += tma_job_units(g, 1);
      } else {
        b.cols[projection_class(c.in_bf16, c.L)].push_back(c);
      }
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
      b.gemms.push_back(a);
    } else {
      const ConvGeom& g = cg[i];
      const int nsplit = x.prec.split_terms;
      const int64_t Kpad = round_up(g.R + 127, 64);
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
  b.insts_off = L.take(sizeof(GemmInst) * (b.gemms.size() + 1));
  int tiles = 0;
  for (const auto& a : b.gemms)
    tiles += static_cast<int>(ceil_div(a.rowsP, 128) * ceil_div(a.rowsQ, 256));
  b.num_tiles = tiles;
  b.tiles_off = L.take(sizeof(GemmTile) * (tiles + 1));
  b.total = L.off;
  return PJ_OK;
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

size_t proj_batch_workspace_size(const pj_batch_desc* descs, int32_t n) {
  Built b;
  if (layout(descs, n, nullptr, &b) != PJ_OK) return 0;
  return b.total;
}

pj_status proj_batch_plan_create(const pj_batch_desc* descs, int32_t n, void* workspace, size_t ws_bytes,
                                 void* stream, pj_batch_plan** plan) {
  if (!plan) return fail(PJ_EINVAL, "plan is NULL");
  *plan = nullptr;
  Built b;
  PJ_TRY(layout(descs, n, nullptr, &b));
  if (!workspace) return fail(PJ_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(PJ_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < b.total) return fail(PJ_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, b.total);
  Built w;
  PJ_TRY(layout(descs, n, workspace, &w));
  int sms = 0;
  PJ_TRY(device_sms(&sms));
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
  // instance table and tile list, longest reduced K first
  std::vector<GemmInst> insts(w.gemms.size());
  std::vector<GemmTile> tiles;
  tiles.reserve(w.num_tiles);
  for (size_t i = 0; i < w.gemms.size(); ++i) {
    if (!build_gemm_inst(w.gemms[i], &insts[i])) return fail(PJ_EINVAL, "could not encode tensor maps for batch entry");
    const GemmInst& I = insts[i];
    for (int ti = 0; ti < static_cast<int>(ceil_div(I.M, 256)); ++ti)
      for (int tj = 0; tj < I.tiles_n; ++tj) tiles.push_back(GemmTile{static_cast<int>(i), ti, tj, I.kc * I.nseg});
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const GemmTile& a, const GemmTile& b) { return a.pad > b.pad; });
  for (int cls = 0; cls < kProjectionClasses; ++cls) {
    PJ_TRY(upload(w.rows[cls], workspace, w.rows_off[cls], st));
    PJ_TRY(upload(w.cols[cls], workspace, w.cols_off[cls], st));
  }
  PJ_TRY(upload(w.sig, workspace, w.sig_off, st));
  PJ_TRY(upload(w.tpl, workspace, w.tpl_off, st));
  // TMA jobs (tensor maps encoded now) and their unit lists, job by job
  std::vector<std::vector<TmaJob>> tma_jobs(kTmaClasses);
  std::vector<std::vector<int4>> tma_units(kTmaClasses);
  for (int tc = 0; tc < kTmaClasses; ++tc) {
    for (size_t j = 0; j < w.tma[tc].size(); ++j) {
      const TmaSpec& sp = w.tma[tc][j];
      TmaJob J;
      if (!make_tma_job(sp.X, sp.ld, sp.in_dtype, sp.cols, sp.g, sp.coef, sp.out, &J))
        return fail(PJ_EINVAL, "could not encode a projection tensor map for a batch entry");
      tma_jobs[tc].push_back(J);
      for (int uy = 0; uy < J.units_y; ++uy)
        for (int ux = 0; ux < J.units_x; ++ux) tma_units[tc].push_back(make_int4(static_cast<int>(j), ux, uy, 0));
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
  PJ_TRY(upload(insts, workspace, w.insts_off, st));
  PJ_TRY(upload(tiles, workspace, w.tiles_off, st));
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
    p->tma_units[tc] = static_cast<int64_t>(tma_units[tc].size());
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
  p->d_insts = ptr<GemmInst>(workspace, w.insts_off);
  p->d_tiles = ptr<GemmTile>(workspace, w.tiles_off);
  p->num_tiles = static_cast<int>(tiles.size());
  p->sms = sms;
  *plan = p;
  return PJ_OK;
}

pj_status proj_batch_run(const pj_batch_plan* plan, void* stream) {
  if (!plan) return fail(PJ_EINVAL, "plan is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PJ_CUDA_TRY(cudaMemsetAsync(plan->ws, 0, sizeof(int), st));
  for (int tc = 0; tc < kTmaClasses; ++tc)
    PJ_CUDA_TRY(launch_project_tma_jobs(tc >= 8, tc % 8 + 1, plan->d_tma_jobs[tc], plan->d_tma_units[tc],
                                        plan->tma_units[tc], static_cast<int*>(plan->ws), plan->sms, st));
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
  PJ_CUDA_TRY(launch_gemm_tc_grouped(plan->d_insts, plan->d_tiles, plan->num_tiles, error_word(plan->ws), plan->sms,
                                     st));
  return PJ_OK;
}

void proj_batch_destroy(pj_batch_plan* plan) { delete plan; }

}  // extern "C"
