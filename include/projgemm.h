/*
 * projgemm.h -- C ABI of the GB300 (sm_103a) library for projection-based
 * GEMM and 1-D cross-correlation (CONV), after Anam, Whatmough and
 * Andreopoulos, "Precision-Energy-Throughput Scaling of Generic Matrix
 * Multiplication and Convolution Kernels via Linear Projections",
 * IEEE TCSVT 24(11), 2014.
 *
 * The method (Sec. III): the inner dimension of every product is cut into
 * blocks (the GEMM subblocks of Sec. II-A, Eq. 2; for CONV the template
 * itself, Sec. II-B).  Each block is split into groups of L consecutive
 * values, each group is projected by an invertible L x L matrix C on one
 * operand and by D = C^-1 on the other (Eq. 5-6, block-diagonal form of
 * Eq. 15), only the first l+1 projections are kept (Eq. 8), the reduced
 * products are formed and accumulated into the output.  R, the number of
 * components kept per block, is (l+1) * ceil(block / L); R equal to the block
 * length reproduces the exact product up to rounding.
 *
 * Conventions for every entry point:
 *  - Matrices are row-major; `ld*` is the row pitch in elements.
 *  - Data pointers are DEVICE pointers owned by the caller; the library never
 *    frees or retains them.  `workspace` is caller-owned device memory of at
 *    least the size the matching *_workspace_size() returns, 256-byte aligned;
 *    its first 256 bytes hold the device error word.  The library allocates no
 *    device memory in these calls.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only
 *    enqueue work; results are ready when the stream is.
 *  - Arguments are validated before anything is enqueued; a violation returns
 *    PJ_EINVAL (or PJ_EUNSUPPORTED for a valid but unimplemented combination)
 *    and enqueues nothing.  pj_last_error() then describes the problem.
 *  - A kernel never traps.  Every wait inside a kernel is bounded; a kernel
 *    that gives up records a code in the device error word and exits, and
 *    pj_check() reports it as PJ_ETIMEOUT.
 *  - There is no CPU fallback: without a usable sm_103a device the compute
 *    entry points return PJ_ECUDA.
 */
#ifndef PROJGEMM_H
#define PROJGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PJ_OK = 0,
  PJ_EINVAL = 1,       /* invalid argument; nothing was enqueued            */
  PJ_EUNSUPPORTED = 2, /* valid but not implemented; nothing was enqueued   */
  PJ_ENOMEM = 3,       /* workspace smaller than *_workspace_size()          */
  PJ_ECUDA = 4,        /* CUDA runtime error (message in pj_last_error)      */
  PJ_ETIMEOUT = 5      /* a kernel gave up a bounded wait (see pj_check)     */
} pj_status;

typedef enum { PJ_F64 = 0, PJ_F32 = 1, PJ_BF16 = 2, PJ_E4M3 = 3 } pj_dtype;

typedef enum {
  PJ_BASIS_DCT2 = 0, /* c[i,j] = cos(pi/L (i+1/2) j), Eq. 7; columns scaled to unit length    */
  PJ_BASIS_HAAR = 1, /* orthonormal multi-level Haar, L a power of two, coarse to fine (Sec. IV) */
  PJ_BASIS_USER = 2  /* any invertible L x L matrix C (Sec. III-B); D = C^-1 (oblique)         */
} pj_basis_kind;

/* Projection basis: kind, group size L, and for PJ_BASIS_USER a HOST pointer
 * (read when the stream runs the call's first copy -- at every replay when the
 * call is captured in a CUDA graph -- so it must stay valid until then)
 * to the L x L row-major matrix C (column j = projection vector j). */
typedef struct {
  int32_t kind;
  int32_t L;
  const double* user_C;
} pj_basis;

/* Arithmetic of the reduced products.
 *  compute:     PJ_F64  -> projections and products in double (CUDA cores);
 *               PJ_BF16 -> projections in FP32, components rounded to BF16,
 *                          products on tcgen05 tensor cores with FP32 accumulation;
 *               PJ_E4M3 -> (the proj_gemm family; correlations through proj_conv and
 *                          batch entries, split_terms 1) projections in FP32, components
 *                          quantised to FP8 E4M3 with one power-of-two (UE8M0) scale
 *                          per 32 consecutive components of a row of A_c or B_d,
 *                          2^ceil(log2(amax/448)) so nothing saturates; block-scaled
 *                          tcgen05 products with FP32 accumulation.
 *  split_terms: 1 = components in plain BF16 (E4M3);
 *               2 = each component x = hi + lo with hi = q(x), lo = q(x - hi), q the
 *                   rounding to BF16 (to E4M3 with its own block scales);
 *                   the product keeps hi*hi + hi*lo + lo*hi (three tensor-core passes).
 *  split_lead:  precision tiering of the kept projections (PJ_BF16 with split_terms = 2,
 *               proj_gemm family only): 0 = every kept projection carries the lo
 *               term; t in [1, l+1) = only projections p < t do (the low-order
 *               projections that hold most of the energy of smooth data), the others
 *               stay plain BF16, so the hi*lo and lo*hi passes shrink to t / (l+1)
 *               of the reduced dimension.
 *  fp8_tier:    precision tiering below the kept projections (proj_gemm family,
 *               PJ_BF16 compute, FP32 output): n > 0 adds the next n projections
 *               of every group, p = l+1 .. l+n (l+1+n <= L), as a correction
 *               computed in FP8 E4M3 with one UE8M0 scale per 32 consecutive
 *               components (one term), accumulated into the same FP32 output.
 *               The result approximates the projection that keeps l+1+n
 *               projections (Eq. 8 with l+n), with the components p > l carried
 *               at E4M3 precision: the incremental reconstruction of Sec. III-A
 *               spent at the lowest precision where the projections hold the
 *               least energy.  0 = none.
 *  Unused fields must be zero. */
typedef struct {
  int32_t compute;
  int32_t split_terms;
  int32_t split_lead;
  int32_t fp8_tier;
} pj_precision;

/* Thread-local description of the last failure in this thread ("" if none). */
const char* pj_last_error(void);

/* Library version string, naming the build variant: "cta-pairs" (reduced GEMMs
 * may run on clusters of two CTAs that share operand tiles by cluster multicast;
 * for one process on one GPU) or "solo" (compiled without any multicast form; the
 * build that processes running one per GPU on several GPUs load). */
const char* pj_version(void);

/* Synchronize `stream`, read and clear the device error word at the start of
 * `workspace`.  Returns PJ_OK, PJ_ETIMEOUT (a kernel gave up a wait) or PJ_ECUDA. */
pj_status pj_check(void* workspace, void* stream);

/* Failure-detection self-test (no counterpart in the paper).  Enqueues a kernel
 * whose bounded waits cannot be satisfied and leaves the code of the wait that
 * gave up in the workspace's error word, so that the caller's pj_check returns
 * PJ_ETIMEOUT:
 *   which = 0: one thread waits on an mbarrier nothing arrives at; another
 *              waiting thread gives up as soon as the error word is set;
 *   which = 1: a 256 x 256 x 1024 BF16 product on one CTA pair (two solo CTAs
 *              in the "solo" build) whose copy
 *              producers stop after two of the 16 K stages: the MMA and epilogue
 *              warps give up their waits, drain the copies and products already
 *              issued, free their tensor memory and exit.
 * Nothing traps or faults and the context stays usable.  Takes about 2 s (the
 * wait limit).  workspace: 256-byte aligned device memory of at least
 * pj_selftest_workspace_size() bytes; its contents are overwritten. */
size_t pj_selftest_workspace_size(void);
pj_status pj_selftest_timeout(int32_t which, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------- report ---
 * A-posteriori report of the product proj_gemm would compute for A, B (no
 * counterpart in the paper; Sec. III-A's truncation made computable).  One pass
 * over A and B on the GPU sums, per inner block b, ||A_b||^2, ||A_b C_R||^2 and
 * ||(|A_b| |C_R|)||^2 (and the same for B with D_R) in double; the stream is then
 * synchronized and the report filled on the host:
 *   alg_flops:   2 M N K' for the reduced products (K' over every pass of the split
 *                or tier) plus 2 (M + N) K (l+1) for the projections;
 *   alg_bytes:   A and B read once (in_dtype), Y written once (out_dtype);
 *   norm_A, norm_B: Frobenius norms;
 *   trunc_bound: sum_b ||A_b (I - P_b)||_F ||(I - P_b) B_b||_F >= ||A B - Y_R||_F,
 *                by Parseval for the orthonormal DCT-II and Haar bases; -1 for
 *                PJ_BASIS_USER (an oblique projector has no Parseval identity);
 *   round_bound: >= ||Y - Y_R||_F for the chosen arithmetic: f ||(|A| |C_R|)||_F
 *                ||(|D_R| |B|)||_F with f the kernels' componentwise forward-error
 *                factor (PJ_F64, PJ_BF16 with or without the split); -1 for PJ_E4M3.
 * Arguments as for proj_gemm (Y is not needed; out_dtype only sizes alg_bytes).
 * workspace: at least proj_gemm_report_workspace_size(K, block_k) bytes. */
typedef struct {
  double alg_flops;
  double alg_bytes;
  double norm_A;
  double norm_B;
  double trunc_bound;
  double round_bound;
} pj_report;

size_t proj_gemm_report_workspace_size(int64_t K, int64_t block_k);

pj_status proj_gemm_report(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                           int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                           const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream, pj_report* rep);

/* ---------------------------------------------------------------- basis ---
 * Builds, on the GPU in FP64, the kept part of the projection pair (Sec. III-A,
 * Eq. 5-7): C_out[i*lp1 + p] = c[i,p] (L x lp1) and D_out[p*L + i] = d[p,i]
 * (lp1 x L), D = C^-1.  DCT-II and Haar columns are scaled to unit length so
 * that D = C^T; a user matrix is inverted by Gauss-Jordan elimination with
 * partial pivoting (PJ_EINVAL if it is singular; reported through pj_check as
 * PJ_EINVAL).  C_out / D_out are device buffers of L*lp1 doubles.  Limits:
 * 1 <= L <= 64 (a power of two for Haar), 1 <= lp1 <= L. */
pj_status pj_basis_build(const pj_basis* basis, int32_t lp1, double* C_out, double* D_out, void* workspace,
                         size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------- GEMM ---
 * Y (M x N) = sum over inner blocks of the reduced products of the projected
 * operands (Sec. III-B; the block partition of Eq. 2):
 *   A_c[i][b, p, g] = sum_t A[i][b*block_k + g*L + t] c[t,p]
 *   B_d[b, p, g][j] = sum_t d[p,t] B[b*block_k + g*L + t][j]
 *   Y = A_c B_d,   p < l+1,   R = (l+1) * ceil(block_k / L) per full block.
 * The last block may be shorter than block_k and its last group shorter than L
 * (zero extension, exact for the product); it keeps the same l+1.
 *   A: M x K (lda >= K), B: K x N (ldb >= N), Y: M x N (ldy >= N).
 *   in_dtype:  PJ_F64 (with compute PJ_F64) or PJ_F32 / PJ_BF16 (compute PJ_BF16 or PJ_E4M3).
 *   out_dtype: PJ_F64 (compute PJ_F64) or PJ_F32 / PJ_BF16.
 *   Requirements: block_k % L == 0, R % (block_k / L) == 0, 1 <= l+1 <= L,
 *   L <= 64, device pointers 16-byte aligned, M, N, K >= 0 (0 -> no work). */
size_t proj_gemm_workspace_size(int64_t M, int64_t N, int64_t K, int64_t block_k, int64_t R,
                                const pj_basis* basis, const pj_precision* prec);

pj_status proj_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, void* Y, int64_t ldy, int64_t M,
                    int64_t N, int64_t K, int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R,
                    const pj_basis* basis, const pj_precision* prec, void* workspace, size_t ws_bytes,
                    void* stream);

/* The two stages of proj_gemm, for timing and for reusing projected operands.
 * proj_gemm_project writes A_c and B_d into `workspace` (either operand may be
 * NULL to keep the copy already there); proj_gemm_multiply forms Y from them.
 * Arguments mean the same as for proj_gemm. */
pj_status proj_gemm_project(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N,
                            int64_t K, int32_t in_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                            const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream);

pj_status proj_gemm_multiply(void* Y, int64_t ldy, int64_t M, int64_t N, int64_t K, int32_t out_dtype,
                             int64_t block_k, int64_t R, const pj_basis* basis, const pj_precision* prec,
                             void* workspace, size_t ws_bytes, void* stream);

/* The projection of A fused into the reduced product (Sec. III-B: the projection
 * done as A's blocks are brought in, Sec. II-A's reordering step): B_d must already
 * be in `workspace` (proj_gemm_project with A = NULL and the same arguments), and
 * each of A's groups is projected inside the GEMM kernel as its tile streams in, so
 * A_c is never written to memory.  Y and every argument mean what they mean for
 * proj_gemm.  Supported: PJ_BF16 compute, split_terms 1 or 2 with every component
 * split (split_lead 0), no FP8 tier, L = 8 and R = block_k (all 8 projections of a
 * group: the precision comes from the split, the energy order from the basis), an
 * even number of 128-row tile columns of B_d (ceil(N / 128) even), A 16-byte
 * aligned with 16-byte row pitch, and the CTA-pair build of the library; otherwise
 * PJ_EUNSUPPORTED and nothing is enqueued (use proj_gemm_multiply after projecting A). */
pj_status proj_gemm_fused(const void* A, int64_t lda, void* Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                          int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R, const pj_basis* basis,
                          const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream);

/* Gradients of Y = A P B with P = blockdiag(C_R D_R), the basis held fixed.
 * The paper gives no gradient; this follows from the block-diagonal projector
 * of Eq. 15 truncated to the first l+1 projections as in Eq. 8 (Sec. III-A):
 * Y = A_c B_d is bilinear in A and B, so each gradient is the reduced product
 * with the other operand's projection, mapped back to samples: 
 *   dA = dY (P B)^T = expand_C(dY B_d^T),   dB = (A P)^T dY = expand_D(A_c^T dY),
 * where expand_C maps components back to samples with C (dA[i][gL+t] =
 * sum_p X[i][(g,p)] c[t,p]) and expand_D with D.  A_c and B_d are recomputed
 * from A and B, not stored.  dY: M x N; dA: M x K (ldda >= K); dB: K x N.
 * Same requirements and dtypes as proj_gemm (F32/BF16 inputs, compute BF16,
 * or F64 throughout). */
size_t proj_gemm_backward_workspace_size(int64_t M, int64_t N, int64_t K, int64_t block_k, int64_t R,
                                         const pj_basis* basis, const pj_precision* prec);

pj_status proj_gemm_backward(const void* A, int64_t lda, const void* B, int64_t ldb, const void* dY, int64_t lddy,
                             void* dA, int64_t ldda, void* dB, int64_t lddb, int64_t M, int64_t N, int64_t K,
                             int32_t in_dtype, int32_t out_dtype, int64_t block_k, int64_t R,
                             const pj_basis* basis, const pj_precision* prec, void* workspace, size_t ws_bytes,
                             void* stream);

/* The same gradients from the projections a forward pass already made: A_c and
 * B_d are read from `fwd_workspace`, the workspace of a proj_gemm call (or of
 * proj_gemm_project with both operands) with the same M, N, K, block_k, R, basis
 * and precision, which must still hold them -- the saved state of the forward,
 * as a training step keeps it; A and B themselves are not read.  Gradients as
 * for proj_gemm_backward (same formula, bit-identical results).  dy_dtype is dY's
 * dtype (PJ_F32 or PJ_BF16 for BF16 compute, PJ_F64 for F64).  `workspace` is a
 * separate buffer of proj_gemm_backward_workspace_size bytes.  Errors:
 * PJ_EINVAL for a NULL or too small fwd_workspace (fewer bytes than
 * proj_gemm_workspace_size for this product) or fwd_workspace == workspace, and
 * every error of proj_gemm_backward; the contents of fwd_workspace are not
 * checked, as for proj_gemm_multiply. */
pj_status proj_gemm_backward_saved(const void* fwd_workspace, size_t fwd_ws_bytes, const void* dY, int64_t lddy,
                                   void* dA, int64_t ldda, void* dB, int64_t lddb, int64_t M, int64_t N, int64_t K,
                                   int32_t dy_dtype, int32_t out_dtype, int64_t block_k, int64_t R,
                                   const pj_basis* basis, const pj_precision* prec, void* workspace, size_t ws_bytes,
                                   void* stream);

/* ----------------------------------------------------------------- CONV ---
 * Valid cross-correlation of one signal with n_templates templates
 * (Sec. II-B with k[m+n], Eq. 3), computed from projected inputs (Sec. III-A,
 * Eq. 11-13 with zero extension in place of the cyclic shift; Sec. III-B):
 *   r[m][t] = sum_{g, p<l+1} (sum_i s[m+gL+i] c[i,p]) (sum_i d[p,i] k_t[gL+i]),
 *   0 <= m <= S - T,  R = (l+1) * T / L.
 * The projection block is the template length (block == T).  All lags are
 * computed (the all-samples option of Sec. III-A).
 *   signal: S values; templates: n_templates x T row-major; out: (S-T+1) x
 *   n_templates row-major.
 *   in_dtype PJ_F32, out_dtype PJ_F32.
 *   Bases: any (DCT-II, Haar, USER) with L dividing T and l+1 a power of two;
 *   Haar is computed in the equivalent box basis of the same kept subspace, any
 *   other basis by projecting the group that starts at every sample.  R <= 4096,
 *   1 <= n_templates <= 64, T <= S.
 *   compute PJ_BF16 (split_terms 1), or PJ_E4M3 (Haar, R % 64 == 0, split_terms
 *   1, PJ_F32 signal): E4M3 components with per-32 UE8M0 block scales, the
 *   projected signal of each lag phase quantised per block of 32 and the
 *   correlation lowered to block-scaled GEMMs (as a batch entry of
 *   proj_batch_*, planned in `workspace` for the call, whose size
 *   proj_conv_workspace_size gives with the same precision); this form
 *   synchronizes `stream` once while it plans and is not for stream capture.
 *   The other CONV calls (staged, host buffers, interpolated, allocation-free)
 *   take PJ_BF16 only. */
size_t proj_conv_workspace_size(int64_t S, int64_t T, int64_t n_templates, int64_t block, int64_t R,
                                const pj_basis* basis, const pj_precision* prec);

pj_status proj_conv(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates, void* out,
                    int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R, const pj_basis* basis,
                    const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream);

/* The two stages of proj_conv: project signal and templates into `workspace`
 * (templates may be NULL to keep the projected copy already there), then
 * form the correlation from the workspace. */
pj_status proj_conv_project(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                            int32_t in_dtype, int64_t block, int64_t R, const pj_basis* basis,
                            const pj_precision* prec, void* workspace, size_t ws_bytes, void* stream);

pj_status proj_conv_correlate(int64_t S, int64_t T, int64_t n_templates, void* out, int32_t out_dtype,
                              int64_t block, int64_t R, const pj_basis* basis, const pj_precision* prec,
                              void* workspace, size_t ws_bytes, void* stream);

/* proj_conv for signal, templates and out in HOST memory (page-locked for the
 * copies to overlap the computation).  The lags are cut into `chunks` ranges
 * (1..64); each is correlated from its slice of the signal exactly as proj_conv
 * computes it, into one of two device buffers in `workspace`, and copied to its
 * rows of `out` on a second stream while the next range is computed.  The call
 * only enqueues work: `out` is complete when `stream` is.  The copy stream and
 * its events are created on the first call of each host thread on each device
 * and kept until the process exits; calls are not meant for stream capture.
 * A bounded wait that runs out is reported by pj_check for the last range only.
 * workspace: device memory of proj_conv_host_workspace_size() bytes. */
size_t proj_conv_host_workspace_size(int64_t S, int64_t T, int64_t n_templates, int64_t block, int64_t R,
                                     const pj_basis* basis, const pj_precision* prec, int32_t chunks);

pj_status proj_conv_host(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                         void* out, int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R,
                         const pj_basis* basis, const pj_precision* prec, int32_t chunks, void* workspace,
                         size_t ws_bytes, void* stream);

/* proj_conv with every step-th lag computed and the lags in between filled
 * from their two computed neighbours (Sec. III-A: omit some results of Eq. 13
 * and interpolate them from neighbouring results; step = 2 computes every other
 * lag and sets each missing one to the average of its two neighbours):
 *   r[m] = r_R[m] for m a multiple of step;
 *   r[m] = ((m1 - m) r_R[m0] + (m - m0) r_R[m1]) / step, m0 = step floor(m/step),
 *          m1 = m0 + step, when m1 <= S - T; otherwise r[m] = r_R[m0].
 * step must be a power of two with step <= T / R (the computed lags are whole
 * phases of the box-projected signal), else PJ_EINVAL / PJ_EUNSUPPORTED; step = 1
 * is proj_conv.  Same workspace as proj_conv. */
pj_status proj_conv_interp(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                           void* out, int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R,
                           const pj_basis* basis, const pj_precision* prec, int32_t step, void* workspace,
                           size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batch ---
 * Each instance is the projected GEMM of Sec. III-B (Eq. 2, 8, 15) or the
 * projected correlation of Sec. III-A (Eq. 11-13); the paper runs one problem
 * at a time and has no batching, so only the grouping is new here.
 * Many uneven projected GEMM and CONV instances in one go: batched projection
 * launches followed by ONE persistent grouped tcgen05 GEMM over the tiles of
 * every instance (the paper's kernels applied to many problems at once; each
 * instance means exactly what proj_gemm / proj_conv mean for it).  A
 * correlation instance is lowered to one GEMM per (phase, template) through a
 * Toeplitz matrix of its projected template.  Tiles run longest reduced K
 * first.  Every call only enqueues work, so a run can be captured in a CUDA
 * graph.
 *   pj_batch_desc: op = PJ_OP_GEMM: A (M x K, lda), B (K x N, ldb), Y (M x N, ldy),
 *                  block = block_k; in PJ_F32/PJ_BF16, out PJ_F32/PJ_BF16;
 *                  prec.compute PJ_BF16 or PJ_E4M3 (the E4M3 instances are
 *                  quantised after the projections and run in a second grouped
 *                  launch of the block-scaled kernel);
 *                  op = PJ_OP_CONV: A = signal (S = M), B = templates (N x T, T = K),
 *                  Y = out ((S-T+1) x N), block = T; PJ_F32 in and out;
 *                  prec.compute PJ_BF16 (split_terms 1 or 2) or PJ_E4M3
 *                  (split_terms 1: "FP8 E4M3 with per-block scales" of Sec.
 *                  III-A's components applied to Eq. 11-13: the projected
 *                  signal of each phase is quantised per block of 32 with one
 *                  UE8M0 scale per block, which every overlapping window of the
 *                  lowering reads as its row scale; each template's Toeplitz
 *                  rows per run of 32; the lowered GEMMs run in the block-scaled
 *                  grouped launch).  Device pointers, caller-owned.
 *   proj_batch_workspace_size: bytes of workspace the plan needs (0 if invalid).
 *   proj_batch_plan_create: validates every entry (PJ_EINVAL / PJ_EUNSUPPORTED
 *     name the entry), lays the plan out in `workspace` (owned by the plan until
 *     proj_batch_destroy), builds the projection bases on the GPU and uploads
 *     the instance and tile tables; synchronizes `stream` once.
 *   proj_batch_run: enqueues the plan's launches on `stream`: one projection
 *     launch per (input dtype, group size) class present for the rows of A and
 *     one for the columns of B, one for the correlation signals, one for the
 *     template Toeplitz matrices, then the grouped GEMM.  The inputs are read
 *     at run time, so new data in the same buffers needs no new plan.
 *   proj_batch_destroy: frees the host-side plan (not the workspace). */
typedef enum { PJ_OP_GEMM = 0, PJ_OP_CONV = 1 } pj_op;

typedef struct {
  int32_t op;
  int32_t in_dtype;
  int32_t out_dtype;
  int32_t reserved;
  const void* A;
  const void* B;
  void* Y;
  int64_t M, N, K;
  int64_t lda, ldb, ldy;
  int64_t block;
  int64_t R;
  pj_basis basis;
  pj_precision prec;
} pj_batch_desc;

typedef struct pj_batch_plan pj_batch_plan;

size_t proj_batch_workspace_size(const pj_batch_desc* descs, int32_t n);

pj_status proj_batch_plan_create(const pj_batch_desc* descs, int32_t n, void* workspace, size_t ws_bytes,
                                 void* stream, pj_batch_plan** plan);

/* Tuning of a plan (NULL or all zero = the defaults used by proj_batch_plan_create).
 * The nearest passage in the paper is Sec. II-A, where the subblock size is
 * chosen by test runs on the target core; here tile heights, K splits and the
 * tile order are chosen per instance by a cost model or by measurement.
 *   schedule:  0 = the cost model splits the reduced dimensions that would set the
 *                  makespan (below); tiles sorted by reduced K, longest first, and
 *                  dealt to the persistent CTAs round-robin, so the tiles of one
 *                  instance run side by side and share their operands in L2;
 *              1 = no cost model: tiles sorted by reduced K and dealt round-robin,
 *                  no splits (with tile_rows = 256, the plain longest-K-first order);
 *              2 = as 0, but each tile goes to the CTA the model sees least loaded
 *                  (longest processing time first).
 *   tile_rows: rows of A_c per GEMM tile (the MMA N): 0 = per instance, the
 *              fewest tiles of at most 256 (E4M3: 240) rows with the least padding;
 *              otherwise a fixed height, a multiple of 32 in [32, 256].
 *   max_split: most pieces an instance's reduced dimension may be cut into
 *              (each piece at least 8 K stages; the pieces' partial products are
 *              added into the instance's output, which must be PJ_F32 and is zeroed
 *              first, so its rounding order changes); 0 = 16, 1 = no split.
 *   us_per_tile, us_per_stage, us_per_out_kb: the cost model of one tile, in
 *              microseconds: fixed, per K stage of a 128 x 256 tile (scaled by the
 *              tile's height) and per KB of output; 0 = built-in values.
 *   solo:      0 = the BF16 products run on pairs of CTAs (clusters of two) that
 *                  take neighbouring tiles of one tile row and share its rows of
 *                  A_c, each loading half and multicasting it to both (the
 *                  "solo" build of the library has no pairs and ignores this);
 *              1 = every CTA loads its own tiles.
 *   Correlation instances always use 256-row tiles and no split.
 * The schedule, splits and tiles are decided when the plan is created. */
typedef struct {
  int32_t schedule;
  int32_t tile_rows;
  int32_t max_split;
  int32_t solo;
  double us_per_tile;
  double us_per_stage;
  double us_per_out_kb;
} pj_batch_tuning;

/* What a plan's tuner decided: tiles of the BF16 and E4M3 grouped launches, the
 * persistent CTAs of the larger launch, instances whose reduced dimension was
 * split, and the cost model's makespan (the most loaded CTA, summed over the two
 * launches) and total (all CTAs), in microseconds. */
typedef struct {
  int32_t gemm_tiles;
  int32_t mx_tiles;
  int32_t ctas;
  int32_t split_instances;
  double model_makespan_us;
  double model_total_us;
} pj_batch_info;

size_t proj_batch_workspace_size_tuned(const pj_batch_desc* descs, int32_t n, const pj_batch_tuning* tuning);

pj_status proj_batch_plan_create_tuned(const pj_batch_desc* descs, int32_t n, const pj_batch_tuning* tuning,
                                       void* workspace, size_t ws_bytes, void* stream, pj_batch_plan** plan);

pj_status proj_batch_plan_info(const pj_batch_plan* plan, pj_batch_info* info);

pj_status proj_batch_run(const pj_batch_plan* plan, void* stream);

void proj_batch_destroy(pj_batch_plan* plan);

/* ------------------------------------------------------- no allocation ---
 * proj_conv_noalloc: proj_conv for callers that cannot allocate device memory,
 * such as a plug-in inside a host application that owns the device allocator,
 * or a latency-critical loop that must not call cudaMalloc (which may
 * synchronize the device).  The paper has no counterpart; it only changes where
 * the scratch memory comes from.
 *   Arguments mean what they mean for proj_conv, minus the workspace: the
 *   scratch is one static device array of 20 MiB (enough for S = 2^20 with
 *   64 templates of 4096 at full R), which every GPU that loads this part of
 *   the library holds until the process exits.  Problems that need more
 *   return PJ_ENOMEM and enqueue nothing.  No device memory is allocated.
 *   The first call in each CUDA context (a device's primary context, and
 *   again after cudaDeviceReset replaced it) looks up the array's address in
 *   that context (cudaGetSymbolAddress) and caches it under the context's ID;
 *   make that first call before any stream capture.
 *   All calls share the one array and it keeps the last call's contents: calls
 *   whose GPU work can overlap (different streams, or threads without
 *   ordering) race and corrupt each other's results, so order them.
 *   A kernel that gives up a bounded wait is not reported here; use proj_conv
 *   with a workspace and pj_check when that matters. */
pj_status proj_conv_noalloc(const void* signal, int64_t S, const void* templates, int64_t T, int64_t n_templates,
                            void* out, int32_t in_dtype, int32_t out_dtype, int64_t block, int64_t R,
                            const pj_basis* basis, const pj_precision* prec, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PROJGEMM_H */
