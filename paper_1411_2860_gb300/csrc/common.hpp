// Shared host/device declarations of the library: status handling, the
// workspace layout and the launchers each translation unit provides.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "projgemm.h"

namespace pj {

// ------------------------------------------------------------- status ---

void set_error(const char* fmt, ...);
pj_status fail(pj_status st, const char* fmt, ...);
pj_status cuda_status(cudaError_t e, const char* what);

#define PJ_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #expr);  \
  } while (0)

#define PJ_TRY(expr)                    \
  do {                                  \
    pj_status s_ = (expr);              \
    if (s_ != PJ_OK) return s_;         \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// abi.cu: validation and bookkeeping shared by the entry points.
struct GemmGeom;
struct ConvGeom;
size_t align_up(size_t x);
bool aligned16(const void* p);
pj_status device_sms(int* sms);
pj_status check_basis(const pj_basis* basis);
pj_status check_prec(const pj_precision* prec);
// The workspace is non-NULL, 256-byte aligned and at least `need` bytes.
pj_status check_ws(void* ws, size_t ws_bytes, size_t need);
// Device SM count, and the error word cleared on `st`.
pj_status begin_call(void* ws, cudaStream_t st, int* sms);
// The basis tables for l+1 = lp1 built into the workspace's basis area on `st`
// (`area`: the basis area of a sub-workspace starting there, NULL = ws; p0: the
// first projection kept).
pj_status stage_basis(const pj_basis* basis, int lp1, void* ws, cudaStream_t st, void* area = nullptr, int p0 = 0);
pj_status gemm_geom(int64_t M, int64_t N, int64_t K, int64_t block_k, int64_t R, const pj_basis* basis,
                    const pj_precision* prec, GemmGeom* g);
pj_status conv_geom(int64_t S, int64_t T, int64_t nt, int64_t block, int64_t R, const pj_basis* basis,
                    const pj_precision* prec, ConvGeom* g);
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------- workspace ---
// Every workspace starts with a 256-byte header (device error word first)
// followed by the basis area; the operand areas follow, each 256-B aligned.

constexpr size_t kHeaderBytes = 256;
constexpr int kMaxL = 64;
// Basis area: the user matrix (staging), full C and D, the kept tables in FP64
// and their FP32 copies; every table is sized for L = kMaxL.
constexpr size_t kTab = kMaxL * kMaxL;
constexpr size_t kBasisBytes = 5 * kTab * sizeof(double) + 3 * kTab * sizeof(float);

struct BasisDev {
  double* U64;   // L x L user matrix staged from the host (PJ_BASIS_USER)
  double* C64;   // L x L, C[i*L + j]
  double* D64;   // L x L
  double* Cs64;  // L x lp1 kept columns of C
  double* Ds64;  // lp1 x L kept rows of D
  float* Cs32;   // L x lp1
  float* Ds32;   // lp1 x L
  float* CsT32;  // lp1 x L: CsT32[p * L + i] = Cs32[i * lp1 + p]
};

inline BasisDev basis_area(void* ws) {
  char* b = static_cast<char*>(ws) + kHeaderBytes;
  BasisDev d;
  d.U64 = reinterpret_cast<double*>(b);
  d.C64 = d.U64 + kTab;
  d.D64 = d.C64 + kTab;
  d.Cs64 = d.D64 + kTab;
  d.Ds64 = d.Cs64 + kTab;
  d.Cs32 = reinterpret_cast<float*>(d.Ds64 + kTab);
  d.Ds32 = d.Cs32 + kTab;
  d.CsT32 = d.Ds32 + kTab;
  return d;
}

inline int* error_word(void* ws) { return static_cast<int*>(ws); }

// ---------------------------------------------------------- launchers ---

// basis.cu: build C, D (FP64) and the kept tables of the lp1 projections from p0
// on into `b` (for PJ_BASIS_USER the matrix must already sit in b.U64).
cudaError_t launch_basis_build(int kind, int L, int lp1, BasisDev b, int* err, cudaStream_t st, int p0 = 0);

// project.cu ------------------------------------------------------------
// Rows of A (M x K, pitch lda, dtype in) -> A_c (M x pitch BF16) and columns
// of B -> B_d (N x pitch BF16): component p of global group gg at column
// gg * lp1 + p of segment hi (offset 0) and lo (offset Kp_pad).
struct GemmGeom {
  int64_t M, N, K, Kb, R;  // R: components of a full block
  int L, lp1;
  int64_t Kp;              // sum of components over all blocks
  int64_t Kp_pad;          // Kp rounded up to 64
  int nsplit;              // BF16 components: 1 (hi) or 2 (hi, lo); always 2 for E4M3 compute
  int compute;             // PJ_F64, PJ_BF16 or PJ_E4M3
  int qsplit;              // E4M3 terms: 1 (hi) or 2 (hi, lo)
  int64_t Kq_pad;          // E4M3: Kp rounded up to 128
  int tl;                  // projections p < tl carry the lo term (tl = lp1: all of them)
  int64_t Kt, Kt_pad;      // lead components (groups * tl) and that rounded up to 64
  int tier;                // FP8 tier: projections lp1 .. lp1 + tier - 1 added in E4M3 (0 = none)
};

// Tiered split: only the first tl of the lp1 projections carry the lo term.
// A row of A_c / B_d is then [hi of every component (Kp_pad) | hi of the lead
// components (Kt_pad) | lo of the lead components (Kt_pad)], lead components
// in group-major order gg * tl + p; otherwise [hi (Kp_pad) | lo (Kp_pad)].
inline bool gemm_tiered(const GemmGeom& g) { return g.nsplit > 1 && g.tl < g.lp1; }
inline int64_t gemm_pitch(const GemmGeom& g) {
  return gemm_tiered(g) ? g.Kp_pad + 2 * g.Kt_pad : g.Kp_pad * g.nsplit;
}

// Projections of A's rows and B's columns to BF16 (either operand may be
// NULL): one TMA-staged persistent launch (project_tma.cu) for the operands
// whose layout suits TMA when L = 8, the per-group kernels of project.cu
// otherwise.
cudaError_t launch_project_pair_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int in_dtype,
                                     const GemmGeom& g, const float* Cs, const float* Ds, uint16_t* Ac,
                                     uint16_t* Bd, int* err, int sms, cudaStream_t st);
cudaError_t launch_project_rows_bf16(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs,
                                     uint16_t* Ac, int* err, int sms, cudaStream_t st);
cudaError_t launch_project_cols_bf16(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds,
                                     uint16_t* Bd, int* err, int sms, cudaStream_t st);
cudaError_t launch_project_rows_simt(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs,
                                     uint16_t* Ac, cudaStream_t st);
cudaError_t launch_project_cols_simt(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds,
                                     uint16_t* Bd, cudaStream_t st);

// Where one operand's E4M3 components and block scales go (gemm_mx.cu, mx.cuh).
struct MxQuantSide {
  const uint16_t* src;
  int64_t src_pitch, Kp_pad, rows;
  uint8_t* dst;
  int64_t dst_pitch, Kq_pad;
  uint8_t* sf;
  int tile_rows, atoms;
  int64_t sf_stages, tiles;
  int qsplit;
  int64_t block0;   // first block of this side in a batched launch
};

// TMA-staged projection jobs (L = 8) of a batched launch: one operand of one
// instance, with its own tensor map (or, for a bulk job, read row by row with
// bulk copies); kept in device memory.  Units (32 x 256 input tiles) are listed
// as int4 {job, ux, uy, 0}, job by job.
struct alignas(128) TmaJob {
  CUtensorMap map;          // input: dims {contiguous, rows}, box {256, 32} (unused by bulk jobs)
  const void* src;          // the operand: rows x inner elements, row pitch ld
  int64_t ld, inner, rows;
  const float* coef;        // kept basis vectors as [q * 8 + t], 16-byte aligned
  uint16_t* out;            // A_c (M x pitch) or B_d (N x pitch)
  int64_t n_out, NG, pitch, Kp_pad, Kt_pad;
  int units_x, units_y, nsplit, cols;   // cols: 1 = columns of B
  int tl;                   // lead projections carrying the lo term (see gemm_tiered)
  MxQuantSide q;            // with an E4M3 launch: where the components and scales go (out unused)
};
// launches per (tiles: TMA, bulk) x (output: BF16, E4M3) x (input dtype) x (l+1 = 1..8):
// class = 32 bulk + 16 e4m3 + 8 bf16_input + l
constexpr int kTmaClasses = 64;
// Whether an operand (inner x rows, pitch ld) can be read by the TMA projection.
bool tma_projection_ok(const void* X, int in_dtype, int64_t inner, int64_t rows, int64_t ld);
// Whether it can be read by the bulk-copy form (any pitch; the base aligned to its element).
bool bulk_projection_ok(const void* X, int in_dtype, int64_t inner, int64_t rows, int64_t ld);
// Appends the units of bulk job J (number `job` of its launch): two int4 per 32 x 256
// tile, {job, ux, uy, a0 | ldm << 4 | rows << 8 | cols << 16} and {address of the
// tile's first element, row pitch in bytes} (64-bit each, low word first); a0 and ldm
// are the address and the pitch mod 16, rows and cols the tile's extent in the operand.
void bulk_job_units(const TmaJob& J, int in_dtype, int job, std::vector<int4>& out);
// Fills J for rows of A (cols = 0: inner = K, rows = M) or columns of B (cols = 1:
// inner = N, rows = K); false if the tensor map cannot be encoded (or, bulk, the
// operand is not element-aligned).
bool make_tma_job(const void* X, int64_t ld, int in_dtype, int cols, const GemmGeom& g, const float* coef,
                  uint16_t* out, TmaJob* J, const MxQuantSide* q = nullptr, bool bulk = false);
int64_t tma_job_units(const GemmGeom& g, int cols);
void tma_job_grid(const GemmGeom& g, int cols, int* units_x, int* units_y);
cudaError_t launch_project_tma_jobs(int in_bf16, int lp1, const TmaJob* jobs, const int4* units, int64_t total,
                                    int* err, int sms, cudaStream_t st, bool quant = false, bool bulk = false);

// Projection jobs: one instance's rows of A or columns of B, for one launch that
// serves many instances (block0 = the job's first block in that launch).
struct RowsJob {
  const void* A;
  uint16_t* Ac;
  const float* Cs;
  int64_t lda, M, K, NG, pitch, Kp_pad, block0, Kt_pad;
  int L, lp1, nsplit, in_bf16, tl;
};
struct ColsJob {
  const void* B;
  uint16_t* Bd;
  const float* Ds;
  int64_t ldb, N, K, NG, pitch, Kp_pad, block0, nbx, Kt_pad;
  int L, lp1, nsplit, in_bf16, tl;
};

// ---- column runs staged through shared memory ------------------------------
// In the transposed (K-major) projection of B the 32 lanes of a warp own 32
// consecutive output rows, and for four consecutive groups each lane holds a
// run of 8 (l+1) bytes (l+1 = 4 or 8) bound for the same offset of its row.
// Stored directly, every 16-byte store of the warp lands on 32 different rows.
// Instead the lanes put their runs, group by group, into a 2 KB staging area per part (hi, lo)
// and then read them back row by row, so each warp store covers 512
// contiguous-per-row bytes.  Byte o of the staging area lives at
// base + (o / 128) * seg_pitch + o % 128: a contiguous buffer has seg_pitch =
// 128; a warp's 128-byte column slice of a TMA tile has the tile's row pitch.
// Chunk k of lane c's run is XOR-swizzled so that both the per-lane writes and
// the per-row reads touch every bank once per quarter warp.
template <int LP1>
__device__ __forceinline__ int run_chunk_off(int c, int k) {
  constexpr int kRun = 8 * LP1, kCh = LP1 / 2, kPer128 = 128 / kRun;
  return c * kRun + 16 * (k ^ ((c / kPer128) & (kCh - 1)));
}

template <int LP1>
__device__ __forceinline__ uint4* run_slot(uint8_t* base, int seg_pitch, int part, int c, int k) {
  const int o = part * 2048 + run_chunk_off<LP1>(c, k);
  return reinterpret_cast<uint4*>(base + (o >> 7) * seg_pitch + (o & 127));
}

// Lane `lane` puts group q (< 4) of its run, components v[0 .. LP1), into part
// `part`: chunk q for l+1 = 8, half q % 2 of chunk q / 2 for l+1 = 4.
template <int LP1>
__device__ __forceinline__ void run_put_group(uint8_t* base, int seg_pitch, int part, int lane, int q,
                                              const uint16_t (&v)[8]) {
  auto w2 = [&](int i) { return uint32_t(v[2 * i]) | (uint32_t(v[2 * i + 1]) << 16); };
  if (LP1 == 8) {
    *run_slot<8>(base, seg_pitch, part, lane, q) = make_uint4(w2(0), w2(1), w2(2), w2(3));
  } else {
    uint8_t* ch = reinterpret_cast<uint8_t*>(run_slot<4>(base, seg_pitch, part, lane, q >> 1));
    *reinterpret_cast<uint2*>(ch + 8 * (q & 1)) = make_uint2(w2(0), w2(1));
  }
}

// The warp writes the staged runs of part `part`: run c goes to out0 + c * pitch
// (16-byte aligned) for c < ncols.  Call after a __syncwarp that follows every
// lane's run_put_group.
template <int LP1>
__device__ __forceinline__ void runs_write(uint8_t* base, int seg_pitch, int part, int lane, uint16_t* out0,
                                           int64_t pitch, int ncols) {
  constexpr int kCh = LP1 / 2;
#pragma unroll
  for (int s = 0; s < kCh; ++s) {
    const int gi = s * 32 + lane, c = gi / kCh, k = gi - c * kCh;
    if (c < ncols)
      *reinterpret_cast<uint4*>(out0 + c * pitch + k * 8) = *run_slot<LP1>(base, seg_pitch, part, c, k);
  }
}

// Stores the split part of one group's components (row = start of the output
// row, gg = global group): the lo terms at [Kp_pad + gg lp1], or with a tiered
// split the lead hi and lo terms at [Kp_pad + gg tl] and [Kp_pad + Kt_pad + gg tl].
// store(dst, v, n) writes v[0..n) at dst.
template <typename Store>
__device__ __forceinline__ void store_split_part(uint16_t* row, int64_t gg, const uint16_t (&hi)[8],
                                                 const uint16_t (&lo)[8], int lp1, int tl, int64_t Kp_pad,
                                                 int64_t Kt_pad, Store store) {
  if (tl >= lp1) {
    store(row + Kp_pad + gg * lp1, lo, lp1);
  } else {
    store(row + Kp_pad + gg * tl, hi, tl);
    store(row + Kp_pad + Kt_pad + gg * tl, lo, tl);
  }
}
RowsJob make_rows_job(const void* A, int64_t lda, int in_dtype, const GemmGeom& g, const float* Cs, uint16_t* Ac);
ColsJob make_cols_job(const void* B, int64_t ldb, int in_dtype, const GemmGeom& g, const float* Ds, uint16_t* Bd);
int64_t rows_job_blocks(const RowsJob& J);
int64_t cols_job_blocks(const ColsJob& J);
// Jobs of one class (input dtype x group size, see projection_class) per launch.
int projection_class(int in_bf16, int L);
constexpr int kProjectionClasses = 4;
// job_of[b] = the job of block b (blocks of job j are [block0_j, block0_{j+1})).
cudaError_t launch_project_rows_jobs(int cls, const RowsJob* jobs, const int* job_of, int64_t blocks, cudaStream_t st);
cudaError_t launch_project_cols_jobs(int cls, const ColsJob* jobs, const int* job_of, int64_t blocks, cudaStream_t st);
// FP64 path: A_c (M x Kp, pitch Kp) and B_d (Kp x N, pitch N), both double.
cudaError_t launch_project_rows_f64(const double* A, int64_t lda, const GemmGeom& g, const double* Cs, double* Ac,
                                    cudaStream_t st);
cudaError_t launch_project_cols_f64(const double* B, int64_t ldb, const GemmGeom& g, const double* Ds, double* Bd,
                                    cudaStream_t st);

// gemm_f64.cu: Y = Ac (M x Kp) * Bd (Kp x N) in double.
cudaError_t launch_gemm_f64(const double* Ac, const double* Bd, double* Y, int64_t ldy, int64_t M, int64_t N,
                            int64_t Kp, cudaStream_t st);

// gemm_tc.cu: Y[m][n] = sum over segments s and k < kdim of Q[m][segQ[s] + k] * P[n][segP[s] + k]
// on tcgen05 (BF16 operands, K-major, row pitch 16-byte multiple; columns at or beyond
// xdim read as zero).  Output FP32 or BF16 with row pitch ldy.
// Expansion of the reduced product back to samples, done in the GEMM epilogue
// for the gradients (group size L = 8, l+1 in {1, 2, 4, 8}):
//   mode 1: the product's columns are reduced components k' = g (l+1) + p (the MMA M
//           side, TMEM lanes): out[i][8 g + t] = sum_p Y[i][k'] coef[t (l+1) + p];
//   mode 2: the product's rows are reduced components (TMEM columns):
//           out[8 g + t][j] = sum_p coef[p 8 + t] Y[k'][j].
// Samples at or beyond K (a short last group) are not written.  coef: device
// table (Cs32 for mode 1, Ds32 for mode 2).  out: FP32 or BF16, rows ld apart,
// 16-byte aligned rows.
struct ExpandArgs {
  int mode = 0;
  int lp1 = 0;
  int out_bf16 = 0;
  int64_t K = 0;
  void* out = nullptr;
  int64_t ld = 0;
  const float* coef = nullptr;
};

struct GemmTcArgs {
  ExpandArgs ex;   // expansion in the epilogue (mode 0: Y is written as it is)
  const uint16_t* Q;
  int64_t ldq, rowsQ;
  const uint16_t* P;
  int64_t ldp, rowsP;
  int64_t xdim, kdim;
  int nseg;
  int64_t segQ[3], segP[3];
  int64_t segK[3] = {0, 0, 0};   // components of each segment (0 = kdim)
  void* Y;
  int64_t ldy;
  int out_dtype;
  // Row-split mode (a lowered correlation): Q is a 128-wide view with q_rows_alloc
  // rows; K chunk k of output row r reads view row r + k/2 at column 64 (k mod 2).
  // Output element (i, j) is sample i*128 + j < conv_limit, at Y[(i*128 + j) * conv_stride].
  int conv_mode = 0;
  int64_t q_rows_alloc = 0, conv_stride = 1, conv_limit = 0;
  int bn = 256;   // rows of Q per tile: a multiple of 32 (64 for an MN-major Q), at most 256
  // MN-major operands: Q (P) is stored transposed, as xdim rows of the reduced
  // dimension by rowsQ (rowsP) contiguous values with pitch ldq (ldp); the tensor
  // cores read it as it is, so no transposed copy is made.
  int mnQ = 0, mnP = 0;
  // Set by launch_gemm_tc_generic: CTA pairs (clusters of two) share each Q tile,
  // each loading half of it for both; the Q tensor map then has half-height boxes.
  int pair = 0;
  // Failure-detection self-test only (pj_selftest_timeout): the copy producer stops
  // after this many K stages, so the waits of the MMA and epilogue warps run out.
  int stall_stage = -1;
};
cudaError_t launch_gemm_tc_generic(const GemmTcArgs& a, int* err, int num_sms, cudaStream_t st);
// gemm_cg2.cu: the same product on 2-SM MMAs (clusters of two CTAs computing 256-row
// tiles; an even number of 128-row P tile columns; not for lowered correlations).
// launch_gemm_tc_generic takes this path by itself whenever it applies.
bool gemm_cg2_eligible(const GemmTcArgs& a, int num_sms);
cudaError_t launch_gemm_cg2(const GemmTcArgs& a, int* err, int num_sms, cudaStream_t st);
// gemm_fused.cu: Y = (A projected inside the kernel) x B_d (already in the workspace),
// for L = 8, l+1 = 8, BF16 components (plain or every component split), an even number
// of 128-row B_d tile columns, A rows 16-byte aligned.
bool gemm_fused_supported(const GemmGeom& g, int in_dtype, const void* A, int64_t lda, int num_sms);
cudaError_t launch_gemm_fused(const void* A, int64_t lda, int in_dtype, const uint16_t* Bd, const GemmGeom& g,
                              const float* Cs, void* Y, int64_t ldy, int out_dtype, int* err, int num_sms,
                              cudaStream_t st);

// Whether a single-instance launch of `tiles` tiles of `stages` K stages each
// should share the stages evenly over all SMs (stream-K; FP32 output zeroed
// first): when the tiles fill less than 90 % of one wave, and every SM still
// gets at least 16 stages.  With a wave or more of tiles, CTAs that start in
// the middle of tiles lose the L2 sharing of operand slices between CTAs that
// run the same K stages side by side, which measured slower than a ragged
// last wave (up to 40 % on the block-scaled kernel).
// Tile height (rows of A_c per tile, a multiple of gran, at most bnmax) for a
// single-instance launch: the height whose whole waves of tiles over the SMs
// finish first, counting each tile as its K stages scaled by its height plus a
// fixed cost of 4 stages.  4096 rows over 152 SMs with 16 tile columns, for
// instance, take 224-row tiles: 304 tiles, exactly two waves.
inline int single_launch_bn(int64_t rows, int64_t tiles_n, int64_t stages, int sms, int gran, int bnmax) {
  int best = bnmax;
  double best_t = 0;
  for (int bn = bnmax; bn >= 64; bn -= gran) {
    const int64_t tiles = (rows + bn - 1) / bn * tiles_n;
    const int64_t waves = (tiles + sms - 1) / sms;
    const double t = static_cast<double>(waves) * (static_cast<double>(stages) * bn / 256.0 + 4.0);
    if (bn == bnmax || t < best_t * 0.99) {
      best = bn;
      best_t = t;
    }
  }
  return best;
}

inline bool use_stream_k(int64_t tiles, int64_t stages, int sms) {
  if (tiles < 1 || stages < 16 || tiles * stages < 16 * static_cast<int64_t>(sms)) return false;
  return static_cast<double>(tiles) < 0.9 * sms;
}

// One instance of the grouped GEMM: tensor maps and output description, laid out
// for the kernel (lives in kernel parameters or in device memory).
struct GemmInst {  // 128-byte aligned through its tensor maps
  CUtensorMap mapP, mapQ, mapY;
  void* Y;
  int64_t ldy;
  int64_t conv_stride, conv_limit;
  int M, N, kc, nseg;     // kc: K stages of all segments together
  int segP[3], segQ[3];
  int segKc[3];           // K stages of each segment
  int tiles_n, out_bf16, tma_out, tma_rows, conv_mode;
  // TMA boxes may store (or add into) tile columns that end at or before this
  // column.  A TMA store writes the whole 16-byte chunk that holds a row's last
  // element, so when a row of Y does not end on a 16-byte boundary the ragged
  // last tile column goes through element-guarded stores instead.
  int tma_cols;
  int bn;   // rows of A_c per tile (MMA N): a multiple of 32, at most 256
  int mnQ, mnP;   // MN-major operands (see GemmTcArgs)
  int ilv;        // three equal segments walked stage by stage (stage kk: segment kk % 3, chunk kk / 3)
};
// One tile of a grouped launch: instance, tile row / column, the range
// [k0, k1) of K stages it multiplies (all kc * nseg stages unless the
// instance's reduced dimension is split), and red = 1 when its partial product
// is added to the output (the output is zeroed first) instead of stored.
struct GemmTile {
  int inst, ti, tj, k0, k1, red, pad0, pad1;   // pad0: pair flags (see launch_gemm_tc_grouped)
};
bool build_gemm_inst(const GemmTcArgs& a, GemmInst* I);
int gemm_tiles_of(const GemmInst& I);
// Tiles of CTA c are tiles[cta_off[c] .. cta_off[c+1]); `ctas` blocks.
// pair: the lists were planned for clusters of two CTAs (2c, 2c + 1), whose tile
// i share their rows of A_c unless flagged (pad0 bit 0: loads its own A_c tile;
// bit 1: a stand-in that writes nothing); every instance then has pair = 1.
cudaError_t launch_gemm_tc_grouped(const GemmInst* insts, const GemmTile* tiles, const int* cta_off, int ctas,
                                   int pair, int* err, cudaStream_t st);

// Forward reduced product: Y (M x N) = A_c * B_d^T with split segments.
cudaError_t launch_gemm_tc(const uint16_t* Ac, const uint16_t* Bd, void* Y, int64_t ldy, int out_dtype,
                           const GemmGeom& g, int* err, int num_sms, cudaStream_t st);

// gemm_mx.cu: E4M3 components with one UE8M0 scale per 32-component K block.
// One side of the quantiser: BF16 hi/lo rows (pitch 2 Kp_pad) -> E4M3 rows
// (pitch Kq_pad * qsplit, lo after Kq_pad) and scale blocks per row tile and
// 128-component stage (tile_rows = 128 with 1 block of 512 bytes for the B_d
// side, 240 with 2 blocks for the A_c side).
// side_q = 1 for A_c (tiles of bn rows, bn <= 240), 0 for B_d (tiles of 128 rows).
constexpr int kMxTileRows = 240;
size_t mx_sf_bytes(int64_t rows, int side_q, int64_t Kq_pad, int qsplit, int bn = kMxTileRows);
MxQuantSide make_mx_side(const uint16_t* src, int64_t Kp_pad, int64_t rows, uint8_t* dst, int64_t Kq_pad, int qsplit,
                         uint8_t* sf, int side_q, int bn = kMxTileRows);
// Either side may be NULL.
cudaError_t launch_quantize_mx(const MxQuantSide* a, const MxQuantSide* b, cudaStream_t st);
// The TMA projection writing E4M3 components and their block scales directly
// (rows: L = 8 and l+1 in {1, 2, 4, 8}; columns: l+1 = 8; row pitches TMA can
// read).  *a_done / *b_done say which sides it took; the caller projects the
// others to BF16 and quantises them (launch_quantize_mx).
bool project_mx_fusable(const GemmGeom& g, int side);
cudaError_t launch_project_pair_mx(const void* A, int64_t lda, const void* B, int64_t ldb, int in_dtype,
                                   const GemmGeom& g, const float* Cs, const float* Ds, const MxQuantSide* qa,
                                   const MxQuantSide* qb, int* err, int sms, cudaStream_t st, bool* a_done,
                                   bool* b_done);
// Batched: sides in device memory, job_of[block] = side of that block.
int64_t mx_side_blocks(const MxQuantSide& a);
cudaError_t launch_quantize_mx_jobs(const MxQuantSide* sides, const int* job_of, int64_t blocks, cudaStream_t st);

struct MxGemmArgs {
  int accum = 0;          // add the product into Y (FP32) instead of storing it
  const uint8_t* Q;   // A_c, rowsQ x pitch E4M3
  const uint8_t* P;   // B_d, rowsP x pitch E4M3
  const uint8_t* sfQ;
  const uint8_t* sfP;
  int64_t rowsQ, rowsP, pitch, Kq_pad;
  int qsplit;
  void* Y;
  int64_t ldy;
  int out_dtype;
  int bn = kMxTileRows;   // rows of Q per tile: a multiple of 16, at most 240
  int pair = 0;           // set by launch_gemm_mx: CTA pairs share the Q tiles (half-height Q boxes)
  // Lowered correlation (conv_mode = 1): Q is a projected signal phase as rows of
  // 128 E4M3 components (q_pitch = 128, q_rows of them), K stage k of output row r
  // reads Q row r + k, and element (r, j) is output sample 128 r + j of the phase,
  // written at Y + (128 r + j) * conv_stride while below conv_limit.  sfQ then
  // holds the scales per tile and stage as the kernel reads them.
  int conv_mode = 0;
  int64_t q_pitch = 0, q_rows = 0;
  int64_t conv_stride = 0, conv_limit = 0;
};
struct MxInst {  // 128-byte aligned through its tensor maps
  CUtensorMap mapP, mapQ, mapY;
  const uint8_t* sfP;
  const uint8_t* sfQ;
  void* Y;
  int64_t ldy, sf_stages;
  int M, N, kc, nseg;
  int segP[3], segQ[3];
  int tiles_n, tiles_m, out_bf16, tma_out;
  int tma_cols;   // as GemmInst::tma_cols
  int bn;   // rows of A_c per tile (MMA N): a multiple of 16, at most 240
  int accum;      // every tile adds its product into Y
  int conv_mode;  // as MxGemmArgs
  int64_t conv_stride, conv_limit;
};
bool build_mx_inst(const MxGemmArgs& a, MxInst* I);
cudaError_t launch_gemm_mx(const MxGemmArgs& a, int* err, int num_sms, cudaStream_t st);
cudaError_t launch_gemm_mx_grouped(const MxInst* insts, const GemmTile* tiles, const int* cta_off, int ctas,
                                   int* err, cudaStream_t st);

// backward.cu -----------------------------------------------------------
cudaError_t launch_convert_bf16(const void* X, int in_dtype, int64_t ldx, int64_t rows, int64_t cols, uint16_t* out,
                                int64_t ldo, cudaStream_t st);
cudaError_t launch_expand_rows(const void* X, int acc_dtype, int64_t ldx, const GemmGeom& g, const void* Cs,
                               void* dA, int out_dtype, int64_t ldda, cudaStream_t st);
cudaError_t launch_expand_cols(const void* X, int acc_dtype, int64_t ldx, const GemmGeom& g, const void* Ds,
                               void* dB, int out_dtype, int64_t lddb, cudaStream_t st);
cudaError_t launch_gemm_f64_strided(const double* A, int64_t sam, int64_t sak, const double* B, int64_t sbk,
                                    int64_t sbn, double* Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                                    cudaStream_t st);

// CONV ----------------------------------------------------------------
// Lags are split as m = phi + PH (beta + NB a), phi < PH, beta < NB: every (phi, beta)
// is a Hankel product over 64-component rows of one phase of the projected signal.
//  - box path (Haar, l+1 a power of two): one component per position, the box sums
//    of Lb = T / R samples; PH = Lb phases, NB = 64, lp1c = 1, 8 shifted copies;
//  - general path (any basis, l+1 a power of two): l+1 components per group start
//    position; PH = L phases, NB = 64 / (l+1), lp1c = l+1, max(1, 8 / (l+1)) copies.
// The copies keep every (phi, beta) row view 16-byte aligned for TMA.
struct ConvGeom {
  int64_t S, T, nt, R;
  int Lb;            // box length T / R (box path; 1 = full R)
  int L, lp1;        // group size and kept projections
  int box;           // 1 = box path, 0 = general path
  int PH, NB;        // phases and row offsets (beta) of the lag split
  int lp1c;          // components per signal position in a phase row
  int ncopy;         // position-shifted copies of the projected signal
  int64_t per;       // PH * NB: lags between consecutive rows of a (phi, beta)
  int64_t lags;      // S - T + 1
  int Kc;            // ceil(R / 64) template chunks (components past R are zero)
  int64_t NA;        // rows of the widest (phi, beta) sub-problem
  int64_t P;         // row pitch (elements) of one phase of the projected signal
  int64_t NRP;       // usable rows per phase (even)
  int tiles_per_sub; // ceil(NA / 512)
};

// Projected signal copies G and (k != NULL) template pairs TP in one launch.  The
// box path also clears the error word *err; the general path reads the kept basis
// tables Cs (L x lp1) and Ds (lp1 x L) and leaves *err alone (the caller clears it
// before the basis is built).
cudaError_t launch_conv_project(const float* s, const float* k, const ConvGeom& g, uint16_t* G, uint16_t* TP,
                                int* err, cudaStream_t st, const float* Cs = nullptr, const float* Ds = nullptr);
// pstep > 1: only the lags that are multiples of pstep (pstep divides Lb).
cudaError_t launch_conv_tc(const uint16_t* G, const uint16_t* TP, float* out, const ConvGeom& g, int* err,
                           int num_sms, cudaStream_t st, int pstep = 1);
// Fills the lags that are not multiples of step from their computed neighbours.
cudaError_t launch_conv_interp(float* out, const ConvGeom& g, int step, cudaStream_t st);

}  // namespace pj
