/*
 * FP64 CPU oracle for projection-based GEMM and 1-D cross-correlation
 * (Anam, Whatmough, Andreopoulos, "Precision-Energy-Throughput Scaling of
 * Generic Matrix Multiplication and Convolution Kernels via Linear
 * Projections", IEEE TCSVT 24(11), 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file;
 * only the tests, the package smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header or table with the CUDA library.
 *
 * Everything is plain double precision, row-major, written for reading:
 * loops follow the paper's order (project, multiply per kept projection,
 * accumulate) and carry no blocking or fusion beyond what the paper states.
 * OpenMP splits independent output rows (lags) across host threads only.
 *
 * Notation (Sec. II-III):  a block of the inner dimension holds `kb` values,
 * split into groups of L consecutive values; the L x L matrix C is any
 * invertible matrix and D = C^{-1} (Eq. 5-6); keeping projections p <= l
 * (lp1 = l+1 of them) gives the truncated reconstruction of Eq. 8, applied
 * group by group through the block-diagonal C_N, D_N of Eq. 15.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_BASIS_DCT2 0
#define OR_BASIS_HAAR 1
#define OR_BASIS_USER 2

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Number of threads an OpenMP parallel region uses with the given request. */
int or_threads(int nthreads) {
#ifdef _OPENMP
    int n = 1;
    set_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Basis (Sec. III-A, Eq. 5-7; Haar per the CONV experiments of Sec. IV).    */
/* C[i*L + j] is c[i,j]; column j is the j-th projection vector.             */
/* ------------------------------------------------------------------------ */

/* D = C^{-1} by Gauss-Jordan elimination with partial pivoting.
 * Returns 0 on success, -1 if C is singular to working precision. */
static int invert(int L, const double *C, double *D) {
    double *a = (double *)malloc(sizeof(double) * (size_t)L * 2 * L);
    if (!a) return -1;
    for (int i = 0; i < L; i++)
        for (int j = 0; j < 2 * L; j++)
            a[i * 2 * L + j] = j < L ? C[i * L + j] : (j - L == i ? 1.0 : 0.0);
    double scale = 0.0;
    for (int i = 0; i < L * L; i++) scale = fmax(scale, fabs(C[i]));
    for (int col = 0; col < L; col++) {
        int piv = col;
        for (int r = col + 1; r < L; r++)
            if (fabs(a[r * 2 * L + col]) > fabs(a[piv * 2 * L + col])) piv = r;
        if (!(fabs(a[piv * 2 * L + col]) > 1e-13 * scale)) { free(a); return -1; }
        if (piv != col)
            for (int j = 0; j < 2 * L; j++) {
                double t = a[col * 2 * L + j];
                a[col * 2 * L + j] = a[piv * 2 * L + j];
                a[piv * 2 * L + j] = t;
            }
        double inv = 1.0 / a[col * 2 * L + col];
        for (int j = 0; j < 2 * L; j++) a[col * 2 * L + j] *= inv;
        for (int r = 0; r < L; r++) {
            if (r == col) continue;
            double f = a[r * 2 * L + col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * L; j++) a[r * 2 * L + j] -= f * a[col * 2 * L + j];
        }
    }
    for (int i = 0; i < L; i++)
        for (int j = 0; j < L; j++) D[i * L + j] = a[i * 2 * L + L + j];
    free(a);
    return 0;
}

/* Build C and D = C^{-1}.
 *  DCT2: c[i,j] = cos(pi/L (i+1/2) j) (Eq. 7), each column scaled to unit
 *        length.  Column scaling leaves every truncated product unchanged
 *        (C E_R C^{-1} does not depend on it) and makes D = C^T.
 *  HAAR: L a power of two; column 0 is constant, then the dyadic Haar
 *        wavelets level by level, coarse to fine, left to right within a
 *        level; each is +1 on its first half, -1 on its second half;
 *        all columns unit length, so D = C^T.
 *  USER: C copied from user_C (row-major L x L), D by Gauss-Jordan.
 * Returns 0 on success, -1 on bad arguments or a singular matrix. */
int or_basis(int kind, int L, const double *user_C, double *C, double *D) {
    if (L < 1) return -1;
    if (kind == OR_BASIS_DCT2) {
        for (int i = 0; i < L; i++)
            for (int j = 0; j < L; j++)
                C[i * L + j] = cos(M_PI / L * (i + 0.5) * j);
    } else if (kind == OR_BASIS_HAAR) {
        if (L & (L - 1)) return -1;
        for (int i = 0; i < L * L; i++) C[i] = 0.0;
        for (int i = 0; i < L; i++) C[i * L + 0] = 1.0;
        int col = 1;
        for (int width = L; width >= 2; width /= 2) {      /* support length */
            for (int start = 0; start < L; start += width) { /* left to right */
                for (int i = 0; i < width; i++)
                    C[(start + i) * L + col] = i < width / 2 ? 1.0 : -1.0;
                col++;
            }
        }
    } else if (kind == OR_BASIS_USER) {
        if (!user_C) return -1;
        memcpy(C, user_C, sizeof(double) * (size_t)L * L);
        return invert(L, C, D);
    } else {
        return -1;
    }
    for (int j = 0; j < L; j++) {
        double n2 = 0.0;
        for (int i = 0; i < L; i++) n2 += C[i * L + j] * C[i * L + j];
        double inv = 1.0 / sqrt(n2);
        for (int i = 0; i < L; i++) C[i * L + j] *= inv;
    }
    for (int i = 0; i < L; i++)
        for (int j = 0; j < L; j++) D[i * L + j] = C[j * L + i];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* GEMM (Sec. II-A Eq. 2; Sec. III-B; Sec. III-C)                           */
/* ------------------------------------------------------------------------ */

/* Y = A B, the plain product of Eq. 2 (A M x K, B K x N). */
void or_gemm_exact(const double *A, const double *B, double *Y,
                   int64_t M, int64_t N, int64_t K, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; i++) {
        double *y = Y + i * N;
        for (int64_t j = 0; j < N; j++) y[j] = 0.0;
        for (int64_t k = 0; k < K; k++) {
            double a = A[i * K + k];
            const double *b = B + k * N;
            for (int64_t j = 0; j < N; j++) y[j] += a * b[j];
        }
    }
}

/* Projected GEMM with lp1 = l+1 kept projections out of L (Sec. III-B).
 * The inner dimension is cut into blocks of Kb (Eq. 2); the last block may
 * be shorter (the "cleanup" border of Sec. II-A) and its last group of L is
 * zero-extended, which leaves every inner product unchanged.  For block n:
 *   A_c[i][g][p] = sum_t A[i][k0+gL+t] c[t,p]      (rows of A times C)
 *   B_d[g][p][j] = sum_t d[p,t] B[k0+gL+t][j]      (D times columns of B)
 * then the (l+1) reduced products A_c[:,:,p] B_d[:,p,:] are accumulated
 * into Y (Eq. 8 applied to every inner product of the block product). */
void or_gemm_proj(const double *A, const double *B, double *Y,
                  int64_t M, int64_t N, int64_t K, int64_t Kb,
                  int L, int lp1, const double *C, const double *D, int nthreads) {
    set_threads(nthreads);
    for (int64_t i = 0; i < M * N; i++) Y[i] = 0.0;
    for (int64_t k0 = 0; k0 < K; k0 += Kb) {
        int64_t kb = K - k0 < Kb ? K - k0 : Kb;
        int64_t G = (kb + L - 1) / L;
        double *Ac = (double *)malloc(sizeof(double) * (size_t)(M * G * lp1));
        double *Bd = (double *)malloc(sizeof(double) * (size_t)(G * lp1 * N));
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < M; i++)
            for (int64_t g = 0; g < G; g++)
                for (int p = 0; p < lp1; p++) {
                    double acc = 0.0;
                    for (int t = 0; t < L; t++) {
                        int64_t k = g * L + t;
                        if (k < kb) acc += A[i * K + k0 + k] * C[t * L + p];
                    }
                    Ac[(i * G + g) * lp1 + p] = acc;
                }
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < G; g++)
            for (int p = 0; p < lp1; p++)
                for (int64_t j = 0; j < N; j++) {
                    double acc = 0.0;
                    for (int t = 0; t < L; t++) {
                        int64_t k = g * L + t;
                        if (k < kb) acc += D[p * L + t] * B[(k0 + k) * N + j];
                    }
                    Bd[(g * lp1 + p) * N + j] = acc;
                }
        for (int p = 0; p < lp1; p++) {       /* one reduced product per projection */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < M; i++)
                for (int64_t g = 0; g < G; g++) {
                    double a = Ac[(i * G + g) * lp1 + p];
                    const double *b = Bd + (g * lp1 + p) * N;
                    double *y = Y + i * N;
                    for (int64_t j = 0; j < N; j++) y[j] += a * b[j];
                }
        }
        free(Ac);
        free(Bd);
    }
}

/* The truncated part of A, block by block:  A_P = A P with
 * P = blockdiag(C_R D_R), i.e. (A_P)[i][k0+gL+t] = sum_{p<lp1} A_c[i][g][p] d[p,t]. */
static void project_rows_back(const double *A, double *AP, int64_t M, int64_t K,
                              int64_t Kb, int L, int lp1, const double *C, const double *D) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; i++)
        for (int64_t k0 = 0; k0 < K; k0 += Kb) {
            int64_t kb = K - k0 < Kb ? K - k0 : Kb;
            for (int64_t g = 0; g * L < kb; g++) {
                double ac[256];
                for (int p = 0; p < lp1; p++) {
                    double acc = 0.0;
                    for (int t = 0; t < L; t++)
                        if (g * L + t < kb) acc += A[i * K + k0 + g * L + t] * C[t * L + p];
                    ac[p] = acc;
                }
                for (int t = 0; t < L; t++) {
                    if (g * L + t >= kb) continue;
                    double acc = 0.0;
                    for (int p = 0; p < lp1; p++) acc += ac[p] * D[p * L + t];
                    AP[i * K + k0 + g * L + t] = acc;
                }
            }
        }
}

/* Closed form of the truncation error:  E = Y - Y_R = (A - A P) B. */
int or_gemm_closed_form(const double *A, const double *B, double *E,
                        int64_t M, int64_t N, int64_t K, int64_t Kb,
                        int L, int lp1, const double *C, const double *D, int nthreads) {
    if (lp1 > 256) return -1;
    set_threads(nthreads);
    double *R = (double *)malloc(sizeof(double) * (size_t)(M * K));
    if (!R) return -1;
    project_rows_back(A, R, M, K, Kb, L, lp1, C, D);
    for (int64_t i = 0; i < M * K; i++) R[i] = A[i] - R[i];
    or_gemm_exact(R, B, E, M, N, K, nthreads);
    free(R);
    return 0;
}

/* Gradients of loss = sum(dY o Y_R) with Y_R = A P B, P = blockdiag(C_R D_R):
 *   dA = dY (P B)^T = dY B^T P^T,     dB = (A P)^T dY = P^T A^T dY.
 * Formed with the dense per-block L x L matrix P (not by re-projecting), so
 * the formula differs from the reduced-product route used on the GPU. */
void or_gemm_adjoint(const double *A, const double *B, const double *dY,
                     double *dA, double *dB, int64_t M, int64_t N, int64_t K,
                     int64_t Kb, int L, int lp1, const double *C, const double *D,
                     int nthreads) {
    set_threads(nthreads);
    double *P = (double *)malloc(sizeof(double) * (size_t)L * L);
    for (int t = 0; t < L; t++)
        for (int u = 0; u < L; u++) {
            double acc = 0.0;
            for (int p = 0; p < lp1; p++) acc += C[t * L + p] * D[p * L + u];
            P[t * L + u] = acc;
        }
    /* PB = P B (block rows), AP = A P (block columns); a short last group
     * keeps only the rows/columns of P that exist. */
    double *PB = (double *)malloc(sizeof(double) * (size_t)(K * N));
    double *AP = (double *)malloc(sizeof(double) * (size_t)(M * K));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < K; k++) {
        int64_t k0 = (k / Kb) * Kb, kb = K - k0 < Kb ? K - k0 : Kb;
        int64_t g = (k - k0) / L, t = (k - k0) % L;
        for (int64_t j = 0; j < N; j++) {
            double acc = 0.0;
            for (int u = 0; u < L; u++)
                if (g * L + u < kb) acc += P[t * L + u] * B[(k0 + g * L + u) * N + j];
            PB[k * N + j] = acc;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; i++)
        for (int64_t k = 0; k < K; k++) {
            int64_t k0 = (k / Kb) * Kb, kb = K - k0 < Kb ? K - k0 : Kb;
            int64_t g = (k - k0) / L, u = (k - k0) % L;
            double acc = 0.0;
            for (int t = 0; t < L; t++)
                if (g * L + t < kb) acc += A[i * K + k0 + g * L + t] * P[t * L + u];
            AP[i * K + k] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; i++)
        for (int64_t k = 0; k < K; k++) {
            double acc = 0.0;
            for (int64_t j = 0; j < N; j++) acc += dY[i * N + j] * PB[k * N + j];
            dA[i * K + k] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < K; k++)
        for (int64_t j = 0; j < N; j++) {
            double acc = 0.0;
            for (int64_t i = 0; i < M; i++) acc += AP[i * K + k] * dY[i * N + j];
            dB[k * N + j] = acc;
        }
    free(P);
    free(PB);
    free(AP);
}

/* Selected entries of the projected product: out[e] = Y_R[ii[e]][jj[e]].
 * Same steps as or_gemm_proj restricted to one row of A and one column of B. */
void or_gemm_proj_entries(const double *A, const double *B, int64_t M, int64_t N,
                          int64_t K, int64_t Kb, int L, int lp1,
                          const double *C, const double *D, const int64_t *ii,
                          const int64_t *jj, int64_t n, double *out, int nthreads) {
    (void)M;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < n; e++) {
        int64_t i = ii[e], j = jj[e];
        double y = 0.0;
        for (int64_t k0 = 0; k0 < K; k0 += Kb) {
            int64_t kb = K - k0 < Kb ? K - k0 : Kb;
            for (int p = 0; p < lp1; p++)
                for (int64_t g = 0; g * L < kb; g++) {
                    double ac = 0.0, bd = 0.0;
                    for (int t = 0; t < L; t++)
                        if (g * L + t < kb) {
                            ac += A[i * K + k0 + g * L + t] * C[t * L + p];
                            bd += D[p * L + t] * B[(k0 + g * L + t) * N + j];
                        }
                    y += ac * bd;
                }
        }
        out[e] = y;
    }
}

/* ------------------------------------------------------------------------ */
/* CONV: valid cross-correlation (Sec. II-B, Eq. 3 with k[m+n]) and its      */
/* projected form (Sec. III-A, Eq. 11-13 with zero extension instead of the */
/* cyclic permutation, applied per group of L as in Sec. III-B).            */
/* ------------------------------------------------------------------------ */

/* r[m][t] = sum_{n<T} s[m+n] k[t][n],  0 <= m <= S-T. */
void or_conv_exact(const double *s, int64_t S, const double *k, int64_t T,
                   int64_t nt, double *r, int nthreads) {
    set_threads(nthreads);
    int64_t lags = S - T + 1;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < lags; m++)
        for (int64_t t = 0; t < nt; t++) {
            double acc = 0.0;
            for (int64_t n = 0; n < T; n++) acc += s[m + n] * k[t * T + n];
            r[m * nt + t] = acc;
        }
}

/* Projected templates:  k_d[t][g][p] = sum_i d[p,i] k[t][gL+i]  (Eq. 12 per group). */
static void project_templates(const double *k, int64_t T, int64_t nt, int L, int lp1,
                              const double *D, double *kd) {
    int64_t G = (T + L - 1) / L;
    for (int64_t t = 0; t < nt; t++)
        for (int64_t g = 0; g < G; g++)
            for (int p = 0; p < lp1; p++) {
                double acc = 0.0;
                for (int i = 0; i < L; i++)
                    if (g * L + i < T) acc += D[p * L + i] * k[t * T + g * L + i];
                kd[(t * G + g) * lp1 + p] = acc;
            }
}

/* One lag of the projected correlation: the window a = s[m .. m+T) is the
 * translated input (Eq. 11, zero-extended), projected per group,
 *   a_c[g][p] = sum_i a[gL+i] c[i,p],
 * and the lag value is the sum over groups and kept projections of
 * a_c[g][p] k_d[t][g][p] (Eq. 13). */
static void proj_lag(const double *s, int64_t m, int64_t T, int64_t nt, int L, int lp1,
                     const double *C, const double *kd, double *ac, double *rrow) {
    int64_t G = (T + L - 1) / L;
    for (int64_t g = 0; g < G; g++)
        for (int p = 0; p < lp1; p++) {
            double acc = 0.0;
            for (int i = 0; i < L; i++)
                if (g * L + i < T) acc += s[m + g * L + i] * C[i * L + p];
            ac[g * lp1 + p] = acc;
        }
    for (int64_t t = 0; t < nt; t++) {
        double acc = 0.0;
        for (int64_t q = 0; q < G * lp1; q++) acc += ac[q] * kd[t * G * lp1 + q];
        rrow[t] = acc;
    }
}

/* Projected valid cross-correlation at all lags (all samples). */
int or_conv_proj(const double *s, int64_t S, const double *k, int64_t T, int64_t nt,
                 int L, int lp1, const double *C, const double *D, double *r,
                 int nthreads) {
    set_threads(nthreads);
    int64_t G = (T + L - 1) / L, lags = S - T + 1;
    double *kd = (double *)malloc(sizeof(double) * (size_t)(nt * G * lp1));
    if (!kd) return -1;
    project_templates(k, T, nt, L, lp1, D, kd);
#pragma omp parallel
    {
        double *ac = (double *)malloc(sizeof(double) * (size_t)(G * lp1));
#pragma omp for schedule(static)
        for (int64_t m = 0; m < lags; m++) proj_lag(s, m, T, nt, L, lp1, C, kd, ac, r + m * nt);
        free(ac);
    }
    free(kd);
    return 0;
}

/* Projected correlation at every step-th lag, the lags in between filled from
 * their two computed neighbours (Sec. III-A: omit some results of Eq. 13 and
 * interpolate them from neighbouring results; step = 2 computes every other
 * result and replaces each missing one by the average of its two neighbours).
 *   computed lags m = 0, step, 2 step, ...: r[m] = r_R[m] as in or_conv_proj;
 *   other lags with m0 = step floor(m / step), m1 = m0 + step:
 *     r[m] = ((m1 - m) r[m0] + (m - m0) r[m1]) / step   if m1 is a lag,
 *     r[m] = r[m0]                                       past the last computed lag
 *   (the paper does not say what happens there; the nearest result is kept). */
int or_conv_proj_interp(const double *s, int64_t S, const double *k, int64_t T, int64_t nt,
                        int L, int lp1, const double *C, const double *D, int64_t step,
                        double *r, int nthreads) {
    if (step < 1) return -1;
    set_threads(nthreads);
    int64_t G = (T + L - 1) / L, lags = S - T + 1;
    double *kd = (double *)malloc(sizeof(double) * (size_t)(nt * G * lp1));
    if (!kd) return -1;
    project_templates(k, T, nt, L, lp1, D, kd);
#pragma omp parallel
    {
        double *ac = (double *)malloc(sizeof(double) * (size_t)(G * lp1));
#pragma omp for schedule(static)
        for (int64_t m = 0; m < lags; m += step) proj_lag(s, m, T, nt, L, lp1, C, kd, ac, r + m * nt);
        free(ac);
    }
    free(kd);
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < lags; m++) {
        int64_t m0 = m - m % step, m1 = m0 + step;
        if (m == m0) continue;
        for (int64_t t = 0; t < nt; t++) {
            if (m1 < lags)
                r[m * nt + t] = ((double)(m1 - m) * r[m0 * nt + t] + (double)(m - m0) * r[m1 * nt + t]) / (double)step;
            else
                r[m * nt + t] = r[m0 * nt + t];
        }
    }
    return 0;
}

/* Projected correlation at selected (lag, template) entries. */
int or_conv_proj_entries(const double *s, int64_t S, const double *k, int64_t T,
                         int64_t nt, int L, int lp1, const double *C, const double *D,
                         const int64_t *mm, const int64_t *tt, int64_t n, double *out,
                         int nthreads) {
    (void)S;
    set_threads(nthreads);
    int64_t G = (T + L - 1) / L;
    double *kd = (double *)malloc(sizeof(double) * (size_t)(nt * G * lp1));
    if (!kd) return -1;
    project_templates(k, T, nt, L, lp1, D, kd);
#pragma omp parallel
    {
        double *ac = (double *)malloc(sizeof(double) * (size_t)(G * lp1));
#pragma omp for schedule(dynamic, 8)
        for (int64_t e = 0; e < n; e++) {
            int64_t m = mm[e], t = tt[e];
            for (int64_t g = 0; g < G; g++)
                for (int p = 0; p < lp1; p++) {
                    double acc = 0.0;
                    for (int i = 0; i < L; i++)
                        if (g * L + i < T) acc += s[m + g * L + i] * C[i * L + p];
                    ac[g * lp1 + p] = acc;
                }
            double acc = 0.0;
            for (int64_t q = 0; q < G * lp1; q++) acc += ac[q] * kd[t * G * lp1 + q];
            out[e] = acc;
        }
        free(ac);
    }
    free(kd);
    return 0;
}

/* Closed form of the CONV truncation error:
 *   r - r_R = < s[m .. m+T), (I - P) k_t >  with P = blockdiag(C_R D_R). */
int or_conv_closed_form(const double *s, int64_t S, const double *k, int64_t T,
                        int64_t nt, int L, int lp1, const double *C, const double *D,
                        double *e, int nthreads) {
    double *P = (double *)malloc(sizeof(double) * (size_t)L * L);
    double *res = (double *)malloc(sizeof(double) * (size_t)(nt * T));
    if (!P || !res) { free(P); free(res); return -1; }
    for (int a = 0; a < L; a++)
        for (int b = 0; b < L; b++) {
            double acc = 0.0;
            for (int p = 0; p < lp1; p++) acc += C[a * L + p] * D[p * L + b];
            P[a * L + b] = acc;
        }
    for (int64_t t = 0; t < nt; t++)
        for (int64_t n = 0; n < T; n++) {
            int64_t g = n / L, a = n % L;
            double acc = 0.0;
            for (int b = 0; b < L; b++)
                if (g * L + b < T) acc += P[a * L + b] * k[t * T + g * L + b];
            res[t * T + n] = k[t * T + n] - acc;
        }
    or_conv_exact(s, S, res, T, nt, e, nthreads);
    free(P);
    free(res);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Projected operands on their own (Sec. III-B, Fig. 5 and Fig. 6 text).     */
/* ------------------------------------------------------------------------ */

/* A_c of every block, row by row: for row i, block b, group g < G_b and
 * projection p < lp1, out[i][off_b + g*lp1 + p] = sum_t A[i][k0+gL+t] c[t,p]
 * where off_b = sum of G_b' * lp1 over earlier blocks.  Returns the row length. */
int64_t or_project_rows(const double *A, int64_t M, int64_t K, int64_t Kb, int L, int lp1,
                        const double *C, double *out) {
    int64_t width = 0;
    for (int64_t k0 = 0; k0 < K; k0 += Kb) {
        int64_t kb = K - k0 < Kb ? K - k0 : Kb;
        width += (kb + L - 1) / L * lp1;
    }
    if (!out) return width;
    for (int64_t i = 0; i < M; i++) {
        int64_t off = 0;
        for (int64_t k0 = 0; k0 < K; k0 += Kb) {
            int64_t kb = K - k0 < Kb ? K - k0 : Kb;
            int64_t G = (kb + L - 1) / L;
            for (int64_t g = 0; g < G; g++)
                for (int p = 0; p < lp1; p++) {
                    double acc = 0.0;
                    for (int t = 0; t < L; t++)
                        if (g * L + t < kb) acc += A[i * K + k0 + g * L + t] * C[t * L + p];
                    out[i * width + off + g * lp1 + p] = acc;
                }
            off += G * lp1;
        }
    }
    return width;
}

/* B_d of every block: out[off_b + g*lp1 + p][j] = sum_t d[p,t] B[k0+gL+t][j]. */
int64_t or_project_cols(const double *B, int64_t K, int64_t N, int64_t Kb, int L, int lp1,
                        const double *D, double *out) {
    int64_t height = 0;
    for (int64_t k0 = 0; k0 < K; k0 += Kb) {
        int64_t kb = K - k0 < Kb ? K - k0 : Kb;
        height += (kb + L - 1) / L * lp1;
    }
    if (!out) return height;
    int64_t off = 0;
    for (int64_t k0 = 0; k0 < K; k0 += Kb) {
        int64_t kb = K - k0 < Kb ? K - k0 : Kb;
        int64_t G = (kb + L - 1) / L;
        for (int64_t g = 0; g < G; g++)
            for (int p = 0; p < lp1; p++)
                for (int64_t j = 0; j < N; j++) {
                    double acc = 0.0;
                    for (int t = 0; t < L; t++)
                        if (g * L + t < kb) acc += D[p * L + t] * B[(k0 + g * L + t) * N + j];
                    out[(off + g * lp1 + p) * N + j] = acc;
                }
        off += G * lp1;
    }
    return height;
}

/* Projected templates on their own: out[t][g*lp1 + p] (Eq. 12 per group). */
int64_t or_project_templates(const double *k, int64_t T, int64_t nt, int L, int lp1,
                             const double *D, double *out) {
    int64_t G = (T + L - 1) / L;
    if (out) project_templates(k, T, nt, L, lp1, D, out);
    return G * lp1;
}
