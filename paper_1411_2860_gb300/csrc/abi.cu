// C ABI entry points: argument validation (before anything is enqueued),
// workspace layout, and the order of kernel launches for each call.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.hpp"
#include "tc.cuh"

namespace pj {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

pj_status fail(pj_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

pj_status cuda_status(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "CUDA error %s (%d) in %s", cudaGetErrorString(e), static_cast<int>(e), what);
  return PJ_ECUDA;
}

// Helpers shared with batch.cu (declared in common.hpp).

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Streaming multiprocessor count of the current device (cached per device).
pj_status device_sms(int* sms) {
  static int cache[64] = {0};
  int dev = 0;
  PJ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PJ_ECUDA, "device ordinal %d out of range", dev);
  if (cache[dev] == 0) {
    int major = 0, minor = 0, n = 0;
    PJ_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    PJ_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    PJ_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    if (major != 10 || minor != 3)
      return fail(PJ_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a only", dev, major, minor);
    cache[dev] = n;
  }
  *sms = cache[dev];
  return PJ_OK;
}

// ------------------------------------------------------------ validation --

pj_status check_basis(const pj_basis* basis) {
  if (!basis) return fail(PJ_EINVAL, "basis is NULL");
  if (basis->L < 1 || basis->L > kMaxL) return fail(PJ_EINVAL, "basis L=%d outside [1, %d]", basis->L, kMaxL);
  switch (basis->kind) {
    case PJ_BASIS_DCT2:
      return PJ_OK;
    case PJ_BASIS_HAAR:
      if (basis->L & (basis->L - 1)) return fail(PJ_EINVAL, "Haar basis needs L a power of two (L=%d)", basis->L);
      return PJ_OK;
    case PJ_BASIS_USER:
      if (!basis->user_C) return fail(PJ_EINVAL, "PJ_BASIS_USER needs user_C");
      return PJ_OK;
    default:
      return fail(PJ_EINVAL, "unknown basis kind %d", basis->kind);
  }
}

pj_status check_prec(const pj_precision* prec) {
  if (!prec) return fail(PJ_EINVAL, "precision is NULL");
  if (prec->compute != PJ_F64 && prec->compute != PJ_BF16 && prec->compute != PJ_E4M3)
    return fail(PJ_EUNSUPPORTED, "compute dtype %d not supported (PJ_F64, PJ_BF16 or PJ_E4M3)", prec->compute);
  if (prec->split_terms != 1 && prec->split_terms != 2)
    return fail(PJ_EINVAL, "split_terms must be 1 or 2 (got %d)", prec->split_terms);
  if (prec->compute == PJ_F64 && prec->split_terms != 1)
    return fail(PJ_EINVAL, "split_terms applies to PJ_BF16 and PJ_E4M3 compute only");
  if (prec->fp8_tier < 0) return fail(PJ_EINVAL, "fp8_tier must be >= 0");
  if (prec->fp8_tier && prec->compute != PJ_BF16)
    return fail(PJ_EUNSUPPORTED, "fp8_tier applies to PJ_BF16 compute (the kept projections in BF16)");
  if (prec->split_lead < 0) return fail(PJ_EINVAL, "split_lead must be >= 0");
  if (prec->split_lead && (prec->compute != PJ_BF16 || prec->split_terms != 2))
    return fail(PJ_EUNSUPPORTED, "split_lead applies to PJ_BF16 compute with split_terms = 2");
  return PJ_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Geometry of a projected GEMM; validates block, R and basis.
pj_status gemm_geom(int64_t M, int64_t N, int64_t K, int64_t block_k, int64_t R, const pj_basis* basis,
                    const pj_precision* prec, GemmGeom* g) {
  PJ_TRY(check_basis(basis));
  PJ_TRY(check_prec(prec));
  if (M < 0 || N < 0 || K < 0) return fail(PJ_EINVAL, "negative size M=%lld N=%lld K=%lld", (long long)M,
                                            (long long)N, (long long)K);
  if (M > INT32_MAX || N > INT32_MAX) return fail(PJ_EUNSUPPORTED, "M and N must fit in 31 bits");
  const int L = basis->L;
  if (block_k < L || block_k % L) return fail(PJ_EINVAL, "block_k=%lld must be a positive multiple of L=%d",
                                              (long long)block_k, L);
  const int64_t GB = block_k / L;
  if (R < 1 || R % GB) return fail(PJ_EINVAL, "R=%lld must be a positive multiple of block_k/L=%lld", (long long)R,
                                   (long long)GB);
  const int64_t lp1 = R / GB;
  if (lp1 > L) return fail(PJ_EINVAL, "R=%lld exceeds block_k=%lld", (long long)R, (long long)block_k);
  if (lp1 + prec->fp8_tier > L)
    return fail(PJ_EINVAL, "l+1=%lld plus fp8_tier=%d exceeds L=%d", (long long)lp1, prec->fp8_tier, L);
  g->M = M;
  g->N = N;
  g->K = K;
  g->Kb = block_k;
  g->R = R;
  g->L = L;
  g->lp1 = static_cast<int>(lp1);
  g->compute = prec->compute;
  // E4M3 components are quantised from BF16 hi + lo pairs of the projection.
  g->nsplit = prec->compute == PJ_E4M3 ? 2 : prec->split_terms;
  g->qsplit = prec->split_terms;
  g->tl = (prec->split_lead > 0 && prec->split_lead < lp1) ? prec->split_lead : static_cast<int>(lp1);
  if (K == 0) {
    g->Kp = 0;
  } else {
    const int64_t nb = ceil_div(K, block_k);
    const int64_t kb_last = K - (nb - 1) * block_k;
    g->Kp = (nb - 1) * R + lp1 * ceil_div(kb_last, L);
  }
  g->Kp_pad = round_up(g->Kp > 0 ? g->Kp : 1, 64);
  g->Kq_pad = round_up(g->Kp > 0 ? g->Kp : 1, 128);
  g->Kt = g->Kp / g->lp1 * g->tl;
  g->Kt_pad = round_up(g->Kt > 0 ? g->Kt : 1, 64);
  g->tier = prec->fp8_tier;
  return PJ_OK;
}

// Geometry of the FP8 tier of g: the projections lp1 .. lp1 + tier - 1 of every
// group, as an E4M3 product with one term (its own R = tier * block_k / L).
static GemmGeom tier_geom(const GemmGeom& g) {
  GemmGeom t = g;
  t.lp1 = g.tier;
  t.R = g.tier * (g.Kb / g.L);
  t.compute = PJ_E4M3;
  t.nsplit = 2;
  t.qsplit = 1;
  t.tl = t.lp1;
  t.tier = 0;
  if (g.K == 0) {
    t.Kp = 0;
  } else {
    const int64_t nb = ceil_div(g.K, g.Kb);
    const int64_t kb_last = g.K - (nb - 1) * g.Kb;
    t.Kp = (nb - 1) * t.R + t.lp1 * ceil_div(kb_last, g.L);
  }
  t.Kp_pad = round_up(t.Kp > 0 ? t.Kp : 1, 64);
  t.Kq_pad = round_up(t.Kp > 0 ? t.Kp : 1, 128);
  t.Kt = t.Kp;
  t.Kt_pad = t.Kp_pad;
  return t;
}

struct GemmWs {
  size_t total;
  size_t off_ac, off_bd;
  size_t off_aq, off_bq, off_sfq, off_sfp;  // E4M3 components and scale blocks
  size_t off_tier;   // FP8 tier: a sub-workspace (header, basis area, E4M3 layout of tier_geom) at this offset
};

GemmWs gemm_ws_layout(const GemmGeom& g, int compute) {
  GemmWs w;
  w.off_tier = 0;
  size_t off = align_up(kHeaderBytes + kBasisBytes);
  if (compute == PJ_F64) {
    w.off_ac = off;
    off = align_up(off + sizeof(double) * g.M * g.Kp);
    w.off_bd = off;
    off = align_up(off + sizeof(double) * g.Kp * g.N);
  } else {
    const size_t pitch = gemm_pitch(g);
    w.off_ac = off;
    off = align_up(off + 2 * pitch * g.M);
    w.off_bd = off;
    off = align_up(off + 2 * pitch * g.N);
    if (compute == PJ_E4M3) {
      const size_t qpitch = g.Kq_pad * g.qsplit;
      w.off_aq = off;
      off = align_up(off + qpitch * g.M);
      w.off_bq = off;
      off = align_up(off + qpitch * g.N);
      w.off_sfq = off;
      off = align_up(off + mx_sf_bytes(g.M, 1, g.Kq_pad, g.qsplit, 64));  // room for tiles of >= 64 rows
      w.off_sfp = off;
      off = align_up(off + mx_sf_bytes(g.N, 0, g.Kq_pad, g.qsplit));
    }
  }
  if (g.tier > 0) {
    w.off_tier = off;
    off += gemm_ws_layout(tier_geom(g), PJ_E4M3).total;
  }
  w.total = off;
  return w;
}

pj_status check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (!ws) return fail(PJ_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(PJ_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < need)
    return fail(PJ_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, need);
  return PJ_OK;
}

pj_status check_gemm_dtypes(int in_dtype, int out_dtype, const pj_precision* prec) {
  if (prec->compute == PJ_F64) {
    if (in_dtype != PJ_F64 || out_dtype != PJ_F64)
      return fail(PJ_EUNSUPPORTED, "PJ_F64 compute takes PJ_F64 input and output");
  } else {
    if (in_dtype != PJ_F32 && in_dtype != PJ_BF16)
      return fail(PJ_EUNSUPPORTED, "PJ_BF16 compute takes PJ_F32 or PJ_BF16 input (got %d)", in_dtype);
    if (out_dtype != PJ_F32 && out_dtype != PJ_BF16)
      return fail(PJ_EUNSUPPORTED, "PJ_BF16 / PJ_E4M3 compute writes PJ_F32 or PJ_BF16 output (got %d)", out_dtype);
  }
  return PJ_OK;
}

pj_status stage_basis(const pj_basis* basis, int lp1, void* ws, cudaStream_t st, void* area, int p0) {
  BasisDev b = basis_area(area ? area : ws);
  if (basis->kind == PJ_BASIS_USER)
    PJ_CUDA_TRY(cudaMemcpyAsync(b.U64, basis->user_C, sizeof(double) * basis->L * basis->L, cudaMemcpyHostToDevice,
                                st));
  PJ_CUDA_TRY(launch_basis_build(basis->kind, basis->L, lp1, b, error_word(ws), st, p0));
  return PJ_OK;
}

pj_status begin_call(void* ws, cudaStream_t st, int* sms) {
  PJ_TRY(device_sms(sms));
  PJ_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(int), st));
  return PJ_OK;
}

// ------------------------------------------------------------------ CONV --

pj_status conv_geom(int64_t S, int64_t T, int64_t nt, int64_t block, int64_t R, const pj_basis* basis,
                    const pj_precision* prec, ConvGeom* g) {
  PJ_TRY(check_basis(basis));
  PJ_TRY(check_prec(prec));
  if (T < 1 || S < T) return fail(PJ_EINVAL, "need 1 <= T <= S (S=%lld, T=%lld)", (long long)S, (long long)T);
  if (nt < 1) return fail(PJ_EINVAL, "n_templates must be >= 1");
  if (block != T) return fail(PJ_EINVAL, "block must equal the template length T (block=%lld, T=%lld)",
                              (long long)block, (long long)T);
  const int L = basis->L;
  if (T % L) return fail(PJ_EINVAL, "T=%lld must be a multiple of L=%d", (long long)T, L);
  if (R < 1 || (R * L) % T) return fail(PJ_EINVAL, "R=%lld must be (l+1)*T/L", (long long)R);
  const int64_t lp1 = R * L / T;
  if (lp1 < 1 || lp1 > L) return fail(PJ_EINVAL, "R=%lld gives l+1=%lld outside [1, L]", (long long)R,
                                      (long long)lp1);
  if (lp1 & (lp1 - 1))
    return fail(PJ_EUNSUPPORTED, "CONV needs l+1 a power of two (its components fill 64-wide rows)");
  if (prec->compute != PJ_BF16 || prec->split_terms != 1 || prec->fp8_tier)
    return fail(PJ_EUNSUPPORTED, "CONV supports PJ_BF16 compute with split_terms = 1 and no FP8 tier");
  if (R > 64 * 64) return fail(PJ_EUNSUPPORTED, "CONV supports R <= 4096");
  if (nt > 64) return fail(PJ_EUNSUPPORTED, "CONV supports at most 64 templates per call");
  if (S > (int64_t(1) << 31)) return fail(PJ_EUNSUPPORTED, "signal longer than 2^31");
  g->S = S;
  g->T = T;
  g->nt = nt;
  g->R = R;
  g->L = L;
  g->lp1 = static_cast<int>(lp1);
  // Haar with l+1 a power of two keeps the functions constant on runs of T / R
  // samples (a power of two): the box path.  Anything else: the general path.
  g->box = basis->kind == PJ_BASIS_HAAR ? 1 : 0;
  g->Lb = g->box ? static_cast<int>(T / R) : 1;
  g->PH = g->box ? g->Lb : L;
  g->NB = g->box ? 64 : static_cast<int>(64 / lp1);
  g->lp1c = g->box ? 1 : static_cast<int>(lp1);
  g->ncopy = g->box ? 8 : (lp1 >= 8 ? 1 : static_cast<int>(8 / lp1));
  g->per = static_cast<int64_t>(g->PH) * g->NB;
  g->lags = S - T + 1;
  g->Kc = static_cast<int>(ceil_div(R, 64));
  g->NA = (g->lags - 1) / g->per + 1;
  g->NRP = round_up(g->NA + g->Kc + 1, 2);
  g->P = 64 * g->NRP + 128;
  g->tiles_per_sub = static_cast<int>(ceil_div(g->NA, 512));
  return PJ_OK;
}

struct ConvWs {
  size_t total, off_g, off_tp;
};

ConvWs conv_ws_layout(const ConvGeom& g) {
  ConvWs w;
  size_t off = align_up(kHeaderBytes + kBasisBytes);
  w.off_g = off;
  off = align_up(off + 2 * static_cast<size_t>(g.ncopy) * g.PH * g.P);
  w.off_tp = off;
  off = align_up(off + 2 * static_cast<size_t>(g.Kc + 1) * 128 * 64);
  w.total = off;
  return w;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

}  // namespace pj

using namespace pj;

extern "C" {

const char* pj_last_error(void) { return g_err; }

// The build variant is part of the string: "cta-pairs" (clusters of two CTAs share
// operand tiles by multicast; one-GPU use) or "solo" (no multicast form compiled in).
const char* pj_version(void) {
#if PJ_CTA_PAIRS
  return "projgemm 0.2 (sm_103a, cta-pairs)";
#else
  return "projgemm 0.2 (sm_103a, solo)";
#endif
}

pj_status pj_check(void* workspace, void* stream) {
  if (!workspace) return fail(PJ_EINVAL, "workspace is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PJ_CUDA_TRY(cudaStreamSynchronize(st));
  int code = 0;
  PJ_CUDA_TRY(cudaMemcpy(&code, workspace, sizeof(int), cudaMemcpyDeviceToHost));
  if (code == DEV_OK) return PJ_OK;
  const int zero = 0;
  PJ_CUDA_TRY(cudaMemcpy(workspace, &zero, sizeof(int), cudaMemcpyHostToDevice));
  if (code == DEV_BAD_ARG) return fail(PJ_EINVAL, "device rejected an argument (singular user basis)");
  return fail(PJ_ETIMEOUT, "a kernel gave up a bounded wait (device code 0x%x)", code);
}

pj_status pj_basis_build(const pj_basis* basis, int32_t lp1, double* C_out, double* D_out, void* workspace,
                         size_t ws_bytes, void* stream) {
  PJ_TRY(check_basis(basis));
  if (lp1 < 1 || lp1 > basis->L) return fail(PJ_EINVAL, "lp1=%d outside [1, L=%d]", lp1, basis->L);
  if (!C_out || !D_out) return fail(PJ_EINVAL, "output tables are NULL");
  PJ_TRY(check_ws(workspace, ws_bytes, align_up(kHeaderBytes + kBasisBytes)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  PJ_TRY(stage_basis(basis, lp1, workspace, st));
  BasisDev b = basis_area(workspace);
  const size_t bytes = sizeof(double) * basis->L * lp1;
  PJ_CUDA_TRY(cudaMemcpyAsync(C_out, b.Cs64, bytes, cudaMemcpyDeviceToDevice, st));
  PJ_CUDA_TRY(cudaMemcpyAsync(D_out, b.Ds64, bytes, cudaMemcpyDeviceToDevice, st));
  return PJ_OK;
}

// ------------------------------------------------------------------ GEMM --

size_t proj_gemm_workspace_size(int64_t M, int64_t N, int64_t K, int64_t block_k, int64_t R, const pj_basis* basis,
                                const pj_precision* prec) {
  GemmGeom g{};
  if (gemm_geom(M, N, K, block_k, R, basis, prec, &g) != PJ_OK) return 0;
  return gemm_ws_layout(g, prec->compute).total;
}

static pj_status gemm_validate(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N,
                               int64_t K, int32_t in_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                               const pj_precision* prec, void* ws, size_t ws_bytes, GemmGeom* g, GemmWs* w) {
  PJ_TRY(gemm_geom(M, N, K, block_k, R, basis, prec, g));
  if (prec->compute == PJ_F64 ? in_dtype != PJ_F64 : (in_dtype != PJ_F32 && in_dtype != PJ_BF16))
    return fail(PJ_EUNSUPPORTED, "input dtype %d does not match compute %d", in_dtype, prec->compute);
  if (M > 0 && K > 0) {
    if (A && lda < K) return fail(PJ_EINVAL, "lda=%lld < K=%lld", (long long)lda, (long long)K);
    if (A && !aligned16(A)) return fail(PJ_EINVAL, "A must be 16-byte aligned");
  }
  if (N > 0 && K > 0) {
    if (B && ldb < N) return fail(PJ_EINVAL, "ldb=%lld < N=%lld", (long long)ldb, (long long)N);
    if (B && !aligned16(B)) return fail(PJ_EINVAL, "B must be 16-byte aligned");
  }
  *w = gemm_ws_layout(*g, prec->compute);
  return check_ws(ws, ws_bytes, w->total);
}

// Tile height of the E4M3 product of a single call (the quantiser lays the A_c
// scale blocks out per tile, so both stages must agree): waves over the SMs.
static int mx_single_bn(const GemmGeom& g, int sms) {
  return single_launch_bn(g.M, ceil_div(g.N, 128), (g.Kq_pad / 128) * (g.qsplit == 1 ? 1 : 3), sms, 16,
                          kMxTileRows);
}

static pj_status gemm_project_impl(const void* A, int64_t lda, const void* B, int64_t ldb, int32_t in_dtype,
                                   const pj_basis* basis, const pj_precision* prec, void* ws, const GemmGeom& g,
                                   const GemmWs& w, int sms, cudaStream_t st) {
  PJ_TRY(stage_basis(basis, g.lp1, ws, st));
  BasisDev b = basis_area(ws);
  if (prec->compute == PJ_F64) {
    if (A) PJ_CUDA_TRY(launch_project_rows_f64(static_cast<const double*>(A), lda, g, b.Cs64, at<double>(ws, w.off_ac), st));
    if (B) PJ_CUDA_TRY(launch_project_cols_f64(static_cast<const double*>(B), ldb, g, b.Ds64, at<double>(ws, w.off_bd), st));
  } else {
    if (prec->compute == PJ_E4M3) {
      const MxQuantSide qa = make_mx_side(at<uint16_t>(ws, w.off_ac), g.Kp_pad, g.M, at<uint8_t>(ws, w.off_aq),
                                          g.Kq_pad, g.qsplit, at<uint8_t>(ws, w.off_sfq), 1, mx_single_bn(g, sms));
      const MxQuantSide qb = make_mx_side(at<uint16_t>(ws, w.off_bd), g.Kp_pad, g.N, at<uint8_t>(ws, w.off_bq),
                                          g.Kq_pad, g.qsplit, at<uint8_t>(ws, w.off_sfp), 0);
      // E4M3 components straight from the projection where it can write them; the
      // other sides go through BF16 hi + lo and the quantiser pass.
      bool a_done = false, b_done = false;
      PJ_CUDA_TRY(launch_project_pair_mx(A, lda, B, ldb, in_dtype, g, b.Cs32, b.Ds32, A ? &qa : nullptr,
                                         B ? &qb : nullptr, error_word(ws), sms, st, &a_done, &b_done));
      const void* A2 = a_done ? nullptr : A;
      const void* B2 = b_done ? nullptr : B;
      if (A2 || B2) {
        PJ_CUDA_TRY(launch_project_pair_bf16(A2, lda, B2, ldb, in_dtype, g, b.Cs32, b.Ds32, at<uint16_t>(ws, w.off_ac),
                                             at<uint16_t>(ws, w.off_bd), error_word(ws), sms, st));
        PJ_CUDA_TRY(launch_quantize_mx(A2 ? &qa : nullptr, B2 ? &qb : nullptr, st));
      }
    } else {
      PJ_CUDA_TRY(launch_project_pair_bf16(A, lda, B, ldb, in_dtype, g, b.Cs32, b.Ds32, at<uint16_t>(ws, w.off_ac),
                                           at<uint16_t>(ws, w.off_bd), error_word(ws), sms, st));
    }
  }
  if (g.tier > 0) {
    // The FP8 tier: projections lp1 .. lp1 + tier - 1 (basis tables from p0 = lp1),
    // projected to BF16 hi + lo and quantised to E4M3 with per-32 block scales.
    void* sub = at<char>(ws, w.off_tier);
    const GemmGeom gt = tier_geom(g);
    const GemmWs wt = gemm_ws_layout(gt, PJ_E4M3);
    PJ_TRY(stage_basis(basis, gt.lp1, ws, st, sub, g.lp1));
    BasisDev bt = basis_area(sub);
    PJ_CUDA_TRY(launch_project_pair_bf16(A, lda, B, ldb, in_dtype, gt, bt.Cs32, bt.Ds32, at<uint16_t>(sub, wt.off_ac),
                                         at<uint16_t>(sub, wt.off_bd), error_word(ws), sms, st));
    const MxQuantSide qa = make_mx_side(at<uint16_t>(sub, wt.off_ac), gt.Kp_pad, gt.M, at<uint8_t>(sub, wt.off_aq),
                                        gt.Kq_pad, 1, at<uint8_t>(sub, wt.off_sfq), 1, mx_single_bn(gt, sms));
    const MxQuantSide qb = make_mx_side(at<uint16_t>(sub, wt.off_bd), gt.Kp_pad, gt.N, at<uint8_t>(sub, wt.off_bq),
                                        gt.Kq_pad, 1, at<uint8_t>(sub, wt.off_sfp), 0);
    PJ_CUDA_TRY(launch_quantize_mx(A ? &qa : nullptr, B ? &qb : nullptr, st));
  }
  return PJ_OK;
}

// E4M3 product of the quantised operands of geometry g in (sub-)workspace ws;
// accum: added into the FP32 output instead of stored.
static pj_status mx_multiply(void* Y, int64_t ldy, int32_t out_dtype, void* ws, int* err, const GemmGeom& g,
                             const GemmWs& w, int sms, cudaStream_t st, int accum) {
  MxGemmArgs a{};
  a.Q = at<uint8_t>(ws, w.off_aq);
  a.P = at<uint8_t>(ws, w.off_bq);
  a.sfQ = at<uint8_t>(ws, w.off_sfq);
  a.sfP = at<uint8_t>(ws, w.off_sfp);
  a.rowsQ = g.M;
  a.rowsP = g.N;
  a.pitch = g.Kq_pad * g.qsplit;
  a.Kq_pad = g.Kq_pad;
  a.qsplit = g.qsplit;
  a.Y = Y;
  a.ldy = ldy;
  a.out_dtype = out_dtype;
  a.bn = mx_single_bn(g, sms);
  a.accum = accum;
  PJ_CUDA_TRY(launch_gemm_mx(a, err, sms, st));
  return PJ_OK;
}

static pj_status gemm_multiply_impl(void* Y, int64_t ldy, int32_t out_dtype, const pj_precision* prec, void* ws,
                                    const GemmGeom& g, const GemmWs& w, int sms, cudaStream_t st) {
  if (g.tier > 0) {
    // the BF16 product of the kept projections, then the FP8 tier added into Y
    GemmGeom g0 = g;
    g0.tier = 0;
    PJ_CUDA_TRY(launch_gemm_tc(at<uint16_t>(ws, w.off_ac), at<uint16_t>(ws, w.off_bd), Y, ldy, out_dtype, g0,
                               error_word(ws), sms, st));
    const GemmGeom gt = tier_geom(g);
    return mx_multiply(Y, ldy, out_dtype, at<char>(ws, w.off_tier), error_word(ws), gt, gemm_ws_layout(gt, PJ_E4M3),
                       sms, st, 1);
  }
  if (prec->compute == PJ_F64) {
    PJ_CUDA_TRY(launch_gemm_f64(at<double>(ws, w.off_ac), at<double>(ws, w.off_bd), static_cast<double*>(Y), ldy,
                                g.M, g.N, g.Kp, st));
  } else if (prec->compute == PJ_E4M3) {
    PJ_TRY(mx_multiply(Y, ldy, out_dtype, ws, error_word(ws), g, w, sms, st, 0));
  } else {
    PJ_CUDA_TRY(launch_gemm_tc(at<uint16_t>(ws, w.off_ac), at<uint16_t>(ws, w.off_bd), Y, ldy, out_dtype, g,
                               error_word(ws), sms, st));
  }
  return PJ_OK;
}

static pj_status zero_output(void* Y, int64_t ldy, int64_t M, int64_t N, int32_t out_dtype, cudaStream_t st) {
  const size_t es = out_dtype == PJ_F64 ? 8 : out_dtype == PJ_F32 ? 4 : 2;
  if (M > 0 && N > 0) PJ_CUDA_TRY(cudaMemset2DAsync(Y, ldy * es, 0, N * es, M, st));
  return PJ_OK;
}

pj_status proj_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, void* Y, int64_t ldy, int64_t M,
                    int64_t N, int64_t K, int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R,
                    const pj_basis* basis, const pj_precision* prec, void* workspace, size_t ws_bytes,
                    void* stream) {
  GemmGeom g{};
  GemmWs w;
  if ((!A && M > 0 && K > 0) || (!B && K > 0 && N > 0) || (!Y && M > 0 && N > 0))
    return fail(PJ_EINVAL, "A, B and Y must be non-NULL for non-empty operands");
  PJ_TRY(gemm_validate(A, lda, B, ldb, M, N, K, in_dtype, block_k, R, basis, prec, workspace, ws_bytes, &g, &w));
  PJ_TRY(check_gemm_dtypes(in_dtype, out_dtype, prec));
  if (g.tier && out_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "fp8_tier adds into an FP32 output (PJ_F32)");
  if (M > 0 && N > 0 && ldy < N) return fail(PJ_EINVAL, "ldy=%lld < N=%lld", (long long)ldy, (long long)N);
  if (Y && !aligned16(Y)) return fail(PJ_EINVAL, "Y must be 16-byte aligned");
  if (M == 0 || N == 0) return PJ_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  if (K == 0) return zero_output(Y, ldy, M, N, out_dtype, st);
  PJ_TRY(gemm_project_impl(A, lda, B, ldb, in_dtype, basis, prec, workspace, g, w, sms, st));
  return gemm_multiply_impl(Y, ldy, out_dtype, prec, workspace, g, w, sms, st);
}

pj_status proj_gemm_project(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                            int32_t in_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                            const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream) {
  GemmGeom g{};
  GemmWs w;
  PJ_TRY(gemm_validate(A, lda, B, ldb, M, N, K, in_dtype, block_k, R, basis, prec, workspace, ws_bytes, &g, &w));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  if (K == 0) return PJ_OK;
  return gemm_project_impl(M > 0 ? A : nullptr, lda, N > 0 ? B : nullptr, ldb, in_dtype, basis, prec, workspace, g,
                           w, sms, st);
}

pj_status proj_gemm_multiply(void* Y, int64_t ldy, int64_t M, int64_t N, int64_t K, int32_t out_dtype,
                             int64_t block_k, int64_t R, const pj_basis* basis, const pj_precision* prec,
                             void* workspace, size_t ws_bytes, void* stream) {
  GemmGeom g{};
  GemmWs w;
  PJ_TRY(gemm_geom(M, N, K, block_k, R, basis, prec, &g));
  w = gemm_ws_layout(g, prec->compute);
  PJ_TRY(check_ws(workspace, ws_bytes, w.total));
  if (!Y) return fail(PJ_EINVAL, "Y is NULL");
  if (prec->compute == PJ_F64 ? out_dtype != PJ_F64 : (out_dtype != PJ_F32 && out_dtype != PJ_BF16))
    return fail(PJ_EUNSUPPORTED, "output dtype %d does not match compute %d", out_dtype, prec->compute);
  if (g.tier && out_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "fp8_tier adds into an FP32 output (PJ_F32)");
  if (M > 0 && N > 0 && ldy < N) return fail(PJ_EINVAL, "ldy=%lld < N=%lld", (long long)ldy, (long long)N);
  if (!aligned16(Y)) return fail(PJ_EINVAL, "Y must be 16-byte aligned");
  if (M == 0 || N == 0) return PJ_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(device_sms(&sms));
  if (K == 0) return zero_output(Y, ldy, M, N, out_dtype, st);
  return gemm_multiply_impl(Y, ldy, out_dtype, prec, workspace, g, w, sms, st);
}

pj_status proj_gemm_fused(const void* A, int64_t lda, void* Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                          int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                          const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream) {
  GemmGeom g{};
  GemmWs w;
  if ((!A && M > 0 && K > 0) || (!Y && M > 0 && N > 0)) return fail(PJ_EINVAL, "A and Y must be non-NULL");
  PJ_TRY(gemm_validate(A, lda, nullptr, 0, M, N, K, in_dtype, block_k, R, basis, prec, workspace, ws_bytes, &g, &w));
  PJ_TRY(check_gemm_dtypes(in_dtype, out_dtype, prec));
  if (prec->compute != PJ_BF16 || gemm_tiered(g) || g.tier)
    return fail(PJ_EUNSUPPORTED, "proj_gemm_fused takes PJ_BF16 compute, plain or with every component split");
  if (g.L != 8 || g.lp1 != 8) return fail(PJ_EUNSUPPORTED, "proj_gemm_fused needs L = 8 and R = block_k (l+1 = 8)");
  if (M > 0 && N > 0 && ldy < N) return fail(PJ_EINVAL, "ldy=%lld < N=%lld", (long long)ldy, (long long)N);
  if (Y && !aligned16(Y)) return fail(PJ_EINVAL, "Y must be 16-byte aligned");
  if (M == 0 || N == 0) return PJ_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(device_sms(&sms));
  if (!gemm_fused_supported(g, in_dtype, A, lda, sms))
    return fail(PJ_EUNSUPPORTED, "proj_gemm_fused needs an even number of 128-row tile columns of B_d (N=%lld), A "
                                 "rows 16-byte aligned and the CTA-pair build", (long long)N);
  PJ_TRY(begin_call(workspace, st, &sms));
  if (K == 0) return zero_output(Y, ldy, M, N, out_dtype, st);
  PJ_TRY(stage_basis(basis, g.lp1, workspace, st));
  BasisDev b = basis_area(workspace);
  PJ_CUDA_TRY(launch_gemm_fused(A, lda, in_dtype, at<uint16_t>(workspace, w.off_bd), g, b.Cs32, Y, ldy, out_dtype,
                                error_word(workspace), sms, st));
  return PJ_OK;
}

struct BwdWs {
  size_t total;
  size_t ac, bd, dyb, dac, dbd;
  int64_t ldm, ldn;
};

static BwdWs bwd_ws_layout(const GemmGeom& g, int compute) {
  BwdWs w{};
  size_t off = align_up(kHeaderBytes + kBasisBytes);
  w.ldm = round_up(g.M > 0 ? g.M : 1, 8);
  w.ldn = round_up(g.N > 0 ? g.N : 1, 8);
  auto take = [&](size_t bytes) {
    const size_t at_ = off;
    off = align_up(off + bytes);
    return at_;
  };
  if (compute == PJ_F64) {
    w.ac = take(8 * g.M * g.Kp);
    w.bd = take(8 * g.Kp * g.N);
    w.dac = take(8 * g.M * g.Kp);
    w.dbd = take(8 * g.Kp * g.N);
  } else {
    w.ac = take(2 * g.M * gemm_pitch(g));
    w.bd = take(2 * g.N * gemm_pitch(g));   // B_d as the forward lays it out: N rows of components
    w.dyb = take(2 * g.M * w.ldn);
    w.dac = take(4 * g.M * g.Kp);
    w.dbd = take(4 * g.Kp * g.N);
  }
  w.total = off;
  return w;
}

size_t proj_gemm_backward_workspace_size(int64_t M, int64_t N, int64_t K, int64_t block_k, int64_t R,
                                         const pj_basis* basis, const pj_precision* prec) {
  GemmGeom g{};
  if (gemm_geom(M, N, K, block_k, R, basis, prec, &g) != PJ_OK) return 0;
  if (prec->split_terms != 1 || prec->compute == PJ_E4M3 || prec->fp8_tier) return 0;
  return bwd_ws_layout(g, prec->compute).total;
}

// The two gradient products and their expansion, from projected operands Ac
// (M x pitch) and Bd (N x pitch) -- computed by the backward itself or saved by
// the forward -- and dY (dy_dtype).  The basis is staged in `workspace`.
static pj_status backward_products(const void* Ac_v, const void* Bd_v, const void* dY, int64_t lddy, int32_t dy_dtype,
                                   void* dA, int64_t ldda, void* dB, int64_t lddb, int32_t out_dtype,
                                   const GemmGeom& g, int compute, const BwdWs& w, void* workspace, int sms,
                                   cudaStream_t st) {
  BasisDev b = basis_area(workspace);
  if (compute == PJ_F64) {
    const double* Ac = static_cast<const double*>(Ac_v);
    const double* Bd = static_cast<const double*>(Bd_v);
    double* dAc = at<double>(workspace, w.dac);
    double* dBd = at<double>(workspace, w.dbd);
    const double* dYd = static_cast<const double*>(dY);
    // dA_c (M x Kp) = dY B_d^T;  dB_d (Kp x N) = A_c^T dY
    PJ_CUDA_TRY(launch_gemm_f64_strided(dYd, lddy, 1, Bd, 1, g.N, dAc, g.Kp, g.M, g.Kp, g.N, st));
    PJ_CUDA_TRY(launch_gemm_f64_strided(Ac, 1, g.Kp, dYd, lddy, 1, dBd, g.N, g.Kp, g.N, g.M, st));
    PJ_CUDA_TRY(launch_expand_rows(dAc, PJ_F64, g.Kp, g, b.Cs64, dA, PJ_F64, ldda, st));
    PJ_CUDA_TRY(launch_expand_cols(dBd, PJ_F64, g.N, g, b.Ds64, dB, PJ_F64, lddb, st));
    return PJ_OK;
  }
  const uint16_t* Ac = static_cast<const uint16_t*>(Ac_v);
  const uint16_t* Bd = static_cast<const uint16_t*>(Bd_v);
  uint16_t* dYb = at<uint16_t>(workspace, w.dyb);
  float* dAc = at<float>(workspace, w.dac);
  float* dBd = at<float>(workspace, w.dbd);
  GemmGeom g1 = g;
  g1.nsplit = 1;
  const int64_t pitch = gemm_pitch(g1);
  // A BF16 dY whose rows are 16-byte aligned feeds both products as it is.
  const bool dy_direct = dy_dtype == PJ_BF16 && aligned16(dY) && lddy % 8 == 0;
  if (!dy_direct) PJ_CUDA_TRY(launch_convert_bf16(dY, dy_dtype, lddy, g.M, g.N, dYb, w.ldn, st));
  const uint16_t* dYq = dy_direct ? static_cast<const uint16_t*>(dY) : dYb;
  const int64_t lddq = dy_direct ? lddy : w.ldn;
  // With L = 8 and l+1 a power of two, each product's epilogue maps its components
  // back to samples (expand_C for dA, expand_D for dB) and writes the gradient
  // itself; otherwise the FP32 reduced gradients go through the expansion kernels.
  const size_t oes = out_dtype == PJ_BF16 ? 2 : 4;
  const bool fuse = g.L == 8 && (g.lp1 == 1 || g.lp1 == 2 || g.lp1 == 4 || g.lp1 == 8) &&
                    (ldda * oes) % 16 == 0 && (lddb * oes) % 16 == 0;
  GemmTcArgs a1{};  // dA_c[i][k'] = sum_j dY[i][j] B_d[k'][j]: B_d read MN-major (N rows of components)
  a1.Q = dYq;
  a1.ldq = lddq;
  a1.rowsQ = g.M;
  a1.P = Bd; a1.ldp = pitch; a1.rowsP = g.Kp; a1.mnP = 1;
  a1.xdim = g.N; a1.kdim = g.N; a1.nseg = 1;
  a1.Y = dAc; a1.ldy = g.Kp; a1.out_dtype = PJ_F32;
  if (fuse) {
    a1.ex.mode = 1;
    a1.ex.lp1 = g.lp1;
    a1.ex.out_bf16 = out_dtype == PJ_BF16;
    a1.ex.K = g.K;
    a1.ex.out = dA;
    a1.ex.ld = ldda;
    a1.ex.coef = b.Cs32;
  }
  // dB_d[k'][j] = sum_i A_c[i][k'] dY[i][j]: both operands are read MN-major
  // (A_c and dY as stored, reduced over their rows), so nothing is transposed.
  GemmTcArgs a2{};
  a2.Q = Ac; a2.ldq = pitch; a2.rowsQ = g.Kp; a2.mnQ = 1;
  a2.P = dYq; a2.ldp = lddq; a2.rowsP = g.N; a2.mnP = 1;
  a2.xdim = g.M; a2.kdim = g.M; a2.nseg = 1;
  a2.Y = dBd; a2.ldy = g.N; a2.out_dtype = PJ_F32;
  if (fuse) {
    a2.ex = a1.ex;
    a2.ex.mode = 2;
    a2.ex.out = dB;
    a2.ex.ld = lddb;
    a2.ex.coef = b.Ds32;
  }
  // (One launch over both products' tiles measured slower: 0.18 against 0.158 ms
  // for the 8192 x 4096 x 4096 layer, the two operand streams sharing L2.)
  PJ_CUDA_TRY(launch_gemm_tc_generic(a1, error_word(workspace), sms, st));
  PJ_CUDA_TRY(launch_gemm_tc_generic(a2, error_word(workspace), sms, st));
  if (!fuse) {
    PJ_CUDA_TRY(launch_expand_rows(dAc, PJ_F32, g.Kp, g, b.Cs32, dA, out_dtype, ldda, st));
    PJ_CUDA_TRY(launch_expand_cols(dBd, PJ_F32, g.N, g, b.Ds32, dB, out_dtype, lddb, st));
  }
  return PJ_OK;
}

static pj_status backward_checks(const GemmGeom& g, const pj_precision* prec, const void* dY, int64_t lddy, void* dA,
                                 int64_t ldda, void* dB, int64_t lddb) {
  if (prec->split_terms != 1) return fail(PJ_EUNSUPPORTED, "the backward supports split_terms = 1");
  if (prec->compute == PJ_E4M3) return fail(PJ_EUNSUPPORTED, "the backward supports PJ_F64 and PJ_BF16 compute");
  if (prec->fp8_tier) return fail(PJ_EUNSUPPORTED, "the backward has no FP8 tier");
  const bool need_a = g.M > 0 && g.K > 0, need_b = g.K > 0 && g.N > 0;
  if ((need_a && !dA) || (need_b && !dB) || (g.M > 0 && g.N > 0 && !dY))
    return fail(PJ_EINVAL, "dY, dA and dB must be non-NULL for non-empty operands");
  if (need_a && ldda < g.K) return fail(PJ_EINVAL, "ldda must be >= K");
  if (need_b && lddb < g.N) return fail(PJ_EINVAL, "lddb must be >= N");
  if (g.M > 0 && g.N > 0 && lddy < g.N) return fail(PJ_EINVAL, "lddy must be >= N");
  for (const void* ptr : {dY, static_cast<const void*>(dA), static_cast<const void*>(dB)})
    if (ptr && !aligned16(ptr)) return fail(PJ_EINVAL, "dY, dA and dB must be 16-byte aligned");
  return PJ_OK;
}

// Both gradients are zero when the product has no outputs.
static pj_status backward_zero(void* dA, int64_t ldda, void* dB, int64_t lddb, const GemmGeom& g, int32_t out_dtype,
                               cudaStream_t st) {
  const size_t es = out_dtype == PJ_F64 ? 8 : out_dtype == PJ_F32 ? 4 : 2;
  if (g.M > 0 && g.K > 0) PJ_CUDA_TRY(cudaMemset2DAsync(dA, ldda * es, 0, g.K * es, g.M, st));
  if (g.K > 0 && g.N > 0) PJ_CUDA_TRY(cudaMemset2DAsync(dB, lddb * es, 0, g.N * es, g.K, st));
  return PJ_OK;
}

pj_status proj_gemm_backward(const void* A, int64_t lda, const void* B, int64_t ldb, const void* dY, int64_t lddy,
                             void* dA, int64_t ldda, void* dB, int64_t lddb, int64_t M, int64_t N, int64_t K,
                             int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R,
                             const pj_basis* basis, const pj_precision* prec, void* workspace, size_t ws_bytes,
                             void* stream) {
  GemmGeom g{};
  PJ_TRY(gemm_geom(M, N, K, block_k, R, basis, prec, &g));
  PJ_TRY(backward_checks(g, prec, dY, lddy, dA, ldda, dB, lddb));
  PJ_TRY(check_gemm_dtypes(in_dtype, out_dtype, prec));
  const bool need_a = M > 0 && K > 0, need_b = K > 0 && N > 0;
  if ((need_a && !A) || (need_b && !B)) return fail(PJ_EINVAL, "A, B, dY, dA and dB must be non-NULL for non-empty operands");
  if (need_a && lda < K) return fail(PJ_EINVAL, "lda and ldda must be >= K");
  if (need_b && ldb < N) return fail(PJ_EINVAL, "ldb and lddb must be >= N");
  for (const void* ptr : {A, B})
    if (ptr && !aligned16(ptr)) return fail(PJ_EINVAL, "A, B, dY, dA and dB must be 16-byte aligned");
  const BwdWs w = bwd_ws_layout(g, prec->compute);
  PJ_TRY(check_ws(workspace, ws_bytes, w.total));
  if (K == 0) return PJ_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  if (M == 0 || N == 0) return backward_zero(dA, ldda, dB, lddb, g, out_dtype, st);
  PJ_TRY(stage_basis(basis, g.lp1, workspace, st));
  BasisDev b = basis_area(workspace);
  if (prec->compute == PJ_F64) {
    double* Ac = at<double>(workspace, w.ac);
    double* Bd = at<double>(workspace, w.bd);
    PJ_CUDA_TRY(launch_project_rows_f64(static_cast<const double*>(A), lda, g, b.Cs64, Ac, st));
    PJ_CUDA_TRY(launch_project_cols_f64(static_cast<const double*>(B), ldb, g, b.Ds64, Bd, st));
    return backward_products(Ac, Bd, dY, lddy, PJ_F64, dA, ldda, dB, lddb, out_dtype, g, PJ_F64, w, workspace, sms,
                             st);
  }
  uint16_t* Ac = at<uint16_t>(workspace, w.ac);
  uint16_t* Bd = at<uint16_t>(workspace, w.bd);
  GemmGeom g1 = g;
  g1.nsplit = 1;
  // A_c (M x Kp_pad) and B_d (N x Kp_pad) exactly as the forward projects them, in one launch
  PJ_CUDA_TRY(launch_project_pair_bf16(A, lda, B, ldb, in_dtype, g1, b.Cs32, b.Ds32, Ac, Bd, error_word(workspace),
                                       sms, st));
  return backward_products(Ac, Bd, dY, lddy, in_dtype, dA, ldda, dB, lddb, out_dtype, g, prec->compute, w, workspace,
                           sms, st);
}

pj_status proj_gemm_backward_saved(const void* fwd_workspace, size_t fwd_ws_bytes, const void* dY, int64_t lddy,
                                   void* dA, int64_t ldda, void* dB, int64_t lddb, int64_t M, int64_t N, int64_t K,
                                   int32_t dy_dtype, int32_t out_dtype, int64_t block_k, int64_t R,
                                   const pj_basis* basis, const pj_precision* prec, void* workspace, size_t ws_bytes,
                                   void* stream) {
  GemmGeom g{};
  PJ_TRY(gemm_geom(M, N, K, block_k, R, basis, prec, &g));
  PJ_TRY(backward_checks(g, prec, dY, lddy, dA, ldda, dB, lddb));
  PJ_TRY(check_gemm_dtypes(dy_dtype, out_dtype, prec));
  // the forward's workspace: A_c and B_d where proj_gemm / proj_gemm_project put them
  const GemmWs fw = gemm_ws_layout(g, prec->compute);
  if (!fwd_workspace) return fail(PJ_EINVAL, "fwd_workspace is NULL");
  if (fwd_ws_bytes < fw.total)
    return fail(PJ_EINVAL, "fwd_workspace holds %zu bytes; the forward of this product needs %zu", fwd_ws_bytes,
                fw.total);
  if (fwd_workspace == workspace) return fail(PJ_EINVAL, "fwd_workspace and workspace must be different buffers");
  const BwdWs w = bwd_ws_layout(g, prec->compute);
  PJ_TRY(check_ws(workspace, ws_bytes, w.total));
  if (K == 0) return PJ_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(begin_call(workspace, st, &sms));
  if (M == 0 || N == 0) return backward_zero(dA, ldda, dB, lddb, g, out_dtype, st);
  PJ_TRY(stage_basis(basis, g.lp1, workspace, st));
  const void* fws = fwd_workspace;
  return backward_products(static_cast<const char*>(fws) + fw.off_ac, static_cast<const char*>(fws) + fw.off_bd, dY,
                           lddy, dy_dtype, dA, ldda, dB, lddb, out_dtype, g, prec->compute, w, workspace, sms, st);
}

// ------------------------------------------------------------------ CONV --

// E4M3 correlation of a single call: the batch's lowered correlation on the
// block-scaled MMA (one instance holding every template), planned in the
// caller's workspace for this call.
static pj_batch_desc conv_e4m3_desc(const void* signal, int64_t S, const void* templates, int64_t T,
                                    int64_t n_templates, void* out, int64_t block, int64_t R, const pj_basis* basis,
                                    const pj_precision* prec) {
  pj_batch_desc d{};
  d.op = PJ_OP_CONV;
  d.in_dtype = PJ_F32;
  d.out_dtype = PJ_F32;
  d.A = signal;
  d.B = templates;
  d.Y = out;
  d.M = S;
  d.N = n_templates;
  d.K = T;
  d.block = block;
  d.R = R;
  d.basis = *basis;
  d.prec = *prec;
  return d;
}

size_t proj_conv_workspace_size(int64_t S, int64_t T, int64_t n_templates, int64_t block, int64_t R,
                                const pj_basis* basis, const pj_precision* prec) {
  if (basis && prec && prec->compute == PJ_E4M3) {
    // sized with stand-in addresses (the plan's layout does not read them)
    void* const stand_in = reinterpret_cast<void*>(static_cast<uintptr_t>(256));
    const pj_batch_desc d = conv_e4m3_desc(stand_in, S, stand_in, T, n_templates, stand_in, block, R, basis, prec);
    return proj_batch_workspace_size(&d, 1);
  }
  ConvGeom g{};
  if (conv_geom(S, T, n_templates, block, R, basis, prec, &g) != PJ_OK) return 0;
  return conv_ws_layout(g).total;
}

static pj_status conv_validate(int64_t S, int64_t T, int64_t nt, int64_t block, int64_t R, const pj_basis* basis,
                               const pj_precision* prec, void* ws, size_t ws_bytes, ConvGeom* g, ConvWs* w) {
  PJ_TRY(conv_geom(S, T, nt, block, R, basis, prec, g));
  *w = conv_ws_layout(*g);
  return check_ws(ws, ws_bytes, w->total);
}

pj_status proj_conv_project(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                            int32_t in_dtype, int64_t block, int64_t R, const pj_basis* basis,
                            const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream) {
  ConvGeom g{};
  ConvWs w;
  if (!signal) return fail(PJ_EINVAL, "signal is NULL");
  if (in_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "CONV takes PJ_F32 input");
  PJ_TRY(conv_validate(S, T, n_templates, block, R, basis, prec, workspace, ws_bytes, &g, &w));
  if (!aligned16(signal) || (templates && !aligned16(templates)))
    return fail(PJ_EINVAL, "signal and templates must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g.box) {
    // The box projection needs no basis table and clears the error word itself (one launch per call).
    PJ_CUDA_TRY(launch_conv_project(static_cast<const float*>(signal), static_cast<const float*>(templates), g,
                                    at<uint16_t>(workspace, w.off_g), at<uint16_t>(workspace, w.off_tp),
                                    error_word(workspace), st));
    return PJ_OK;
  }
  // General basis: the kept columns of C (signal) and rows of D (templates) first.
  PJ_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(int), st));
  PJ_TRY(stage_basis(basis, g.lp1, workspace, st));
  BasisDev b = basis_area(workspace);
  PJ_CUDA_TRY(launch_conv_project(static_cast<const float*>(signal), static_cast<const float*>(templates), g,
                                  at<uint16_t>(workspace, w.off_g), at<uint16_t>(workspace, w.off_tp),
                                  error_word(workspace), st, b.Cs32, b.Ds32));
  return PJ_OK;
}

pj_status proj_conv_correlate(int64_t S, int64_t T, int64_t n_templates, void* out, int32_t out_dtype, int64_t block,
                              int64_t R, const pj_basis* basis, const pj_precision* prec, void* workspace,
                              size_t ws_bytes, void* stream) {
  ConvGeom g{};
  ConvWs w;
  if (!out) return fail(PJ_EINVAL, "out is NULL");
  if (out_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "CONV writes PJ_F32 output");
  PJ_TRY(conv_validate(S, T, n_templates, block, R, basis, prec, workspace, ws_bytes, &g, &w));
  if (!aligned16(out)) return fail(PJ_EINVAL, "out must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(device_sms(&sms));
  PJ_CUDA_TRY(launch_conv_tc(at<uint16_t>(workspace, w.off_g), at<uint16_t>(workspace, w.off_tp),
                             static_cast<float*>(out), g, error_word(workspace), sms, st));
  return PJ_OK;
}

pj_status proj_conv_interp(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                           void* out, int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R,
                           const pj_basis* basis, const pj_precision* prec, int32_t step, void* workspace,
                           size_t ws_bytes, void* stream) {
  if (!templates) return fail(PJ_EINVAL, "templates is NULL");
  if (!out) return fail(PJ_EINVAL, "out is NULL");
  if (out_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "CONV writes PJ_F32 output");
  ConvGeom g{};
  ConvWs w;
  PJ_TRY(conv_validate(S, T, n_templates, block, R, basis, prec, workspace, ws_bytes, &g, &w));
  if (step < 1 || (step & (step - 1))) return fail(PJ_EINVAL, "step=%d must be a power of two", step);
  if (step > g.PH || g.PH % step)
    return fail(PJ_EUNSUPPORTED, "step=%d must divide the %d phases the lags are computed in (T/R for the Haar "
                                 "box path, L otherwise)", step, g.PH);
  if (!aligned16(out)) return fail(PJ_EINVAL, "out must be 16-byte aligned");
  PJ_TRY(proj_conv_project(signal, S, templates, T, n_templates, in_dtype, block, R, basis, prec, workspace,
                           ws_bytes, stream));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PJ_TRY(device_sms(&sms));
  PJ_CUDA_TRY(launch_conv_tc(at<uint16_t>(workspace, w.off_g), at<uint16_t>(workspace, w.off_tp),
                             static_cast<float*>(out), g, error_word(workspace), sms, st, step));
  PJ_CUDA_TRY(launch_conv_interp(static_cast<float*>(out), g, step, st));
  return PJ_OK;
}

pj_status proj_conv(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates, void* out,
                    int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R, const pj_basis* basis,
                    const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream) {
  if (!templates) return fail(PJ_EINVAL, "templates is NULL");
  if (!out) return fail(PJ_EINVAL, "out is NULL");
  if (out_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "CONV writes PJ_F32 output");
  if (basis && prec && prec->compute == PJ_E4M3) {
    if (!signal) return fail(PJ_EINVAL, "signal is NULL");
    if (in_dtype != PJ_F32) return fail(PJ_EUNSUPPORTED, "E4M3 CONV takes a PJ_F32 signal and templates");
    const pj_batch_desc d = conv_e4m3_desc(signal, S, templates, T, n_templates, out, block, R, basis, prec);
    pj_batch_plan* plan = nullptr;
    PJ_TRY(proj_batch_plan_create(&d, 1, workspace, ws_bytes, stream, &plan));
    const pj_status st = proj_batch_run(plan, stream);
    proj_batch_destroy(plan);
    return st;
  }
  ConvGeom g{};
  ConvWs w;
  PJ_TRY(conv_validate(S, T, n_templates, block, R, basis, prec, workspace, ws_bytes, &g, &w));
  if (!aligned16(out)) return fail(PJ_EINVAL, "out must be 16-byte aligned");
  PJ_TRY(proj_conv_project(signal, S, templates, T, n_templates, in_dtype, block, R, basis, prec, workspace,
                           ws_bytes, stream));
  return proj_conv_correlate(S, T, n_templates, out, out_dtype, block, R, basis, prec, workspace, ws_bytes, stream);
}

}  // extern "C"
