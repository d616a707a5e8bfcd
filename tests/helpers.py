"""Test-side error bounds for comparing the CUDA path with the FP64 oracle.

The GPU rounds projected components to BF16 (unit roundoff u = 2^-8),
accumulates the reduced products in FP32 (u32 = 2^-24) and forms the
projections themselves in FP32.  For one output the standard forward bound
for an inner product of rounded operands (Higham, Accuracy and Stability of
Numerical Algorithms, Sec. 3.1) gives

  |y_gpu - y_R| <= [ (2u + u^2) + 2 gamma_L (1+u)^2 + 2 gamma_K' (1+u)^2 ] * sum_k |a_k| |b_k|

where a_k, b_k are the exact projected components, |a_k| <= sum_t |A||C| and
gamma_n = n u32 / (1 - n u32).  The factor 2 on gamma_K' allows the tensor
core's accumulation to round toward zero instead of to nearest.  With split
components (x = hi + lo, three products) the first term becomes 4 u^2.
These bounds are computed here from the inputs and the oracle's basis only.
"""
import numpy as np

U_BF16 = 2.0 ** -8
U_F32 = 2.0 ** -24


def gamma(n, u=U_F32):
    return n * u / (1.0 - n * u)


def factor(Kp, L, split=1):
    lead = 4 * U_BF16 ** 2 if split == 2 else 2 * U_BF16 + U_BF16 ** 2
    return lead + 2 * gamma(L) * (1 + U_BF16) ** 2 + 2 * gamma(Kp) * (1 + U_BF16) ** 2


# E4M3 components (the FP8 path): each run of 32 consecutive components of a
# row of A_c or B_d has a power-of-two scale s < 2 m / 448 (m = the run's
# largest magnitude), and rounding to nearest E4M3 (3 mantissa bits) gives
# |q(x) - x| <= u_e |x| + 2^-10 s with u_e = 2^-4 (the second term covers the
# subnormal range).  With two terms, hi = q(x) and lo = q(x - hi) with scales of
# its own, |hi + lo - x| <= 2^-8 |x| + 2^-14 s + 2^-10 s_lo, and the dropped
# product lo*lo adds at most 2^-8 |a| |b| plus terms of the same small kind.
# The components entering the quantiser are BF16 hi + lo pairs (2^-16
# relative).  Per output this gives
#   |y_gpu - y_R| <= [lead + 2 gamma_L (1+u)^2 + 2 gamma_K' (1+u)^2] sum |a_k||b_k|
#                    + v (1+u) (m_a sum_k |b_k| + m_b sum_k |a_k|) + v^2 K' m_a m_b
# with lead = 2 u_e + u_e^2 (plain) or 4 * 2^-8 (two terms), plus 2 * 2^-16,
# v = 2^-10 / 224 (plain) or 2 * 2^-14 / 224 * 1.01 (two terms), and m_a, m_b
# the largest component bounds of the row of A_c and of the column of B_d.
U_E4M3 = 2.0 ** -4


def factor_e4m3(Kp, L, split=1):
    u = U_E4M3 if split == 1 else 2.0 ** -8
    lead = (2 * U_E4M3 + U_E4M3 ** 2) if split == 1 else 4 * 2.0 ** -8
    lead += 2 * 2.0 ** -16
    return lead + 2 * gamma(L) * (1 + u) ** 2 + 2 * gamma(Kp) * (1 + u) ** 2


def e4m3_scale_term(absAc, absBd, split=1):
    """The block-scale (subnormal) part of the E4M3 bound, per output."""
    u = U_E4M3 if split == 1 else 2.0 ** -8
    v = 2.0 ** -10 / 224 if split == 1 else 2 * 2.0 ** -14 / 224 * 1.01
    ma = absAc.max(axis=1)[:, None]
    mb = absBd.max(axis=0)[None, :]
    Kp = absAc.shape[1]
    return v * (1 + u) * (ma * absBd.sum(axis=0)[None, :] + mb * absAc.sum(axis=1)[:, None]) + v * v * Kp * ma * mb


def gemm_abs_parts(A, B, L, C, D, lp1):
    """Componentwise bounds |a_k| <= (|A||C|) and |b_k| <= (|D||B|), group-major."""
    A = np.abs(np.asarray(A, dtype=np.float64))
    B = np.abs(np.asarray(B, dtype=np.float64))
    m, K = A.shape
    NG = -(-K // L)
    Ap = np.zeros((m, NG * L))
    Ap[:, :K] = A
    Bp = np.zeros((NG * L, B.shape[1]))
    Bp[:K] = B
    Ca = np.abs(C[:, :lp1])
    Da = np.abs(D[:lp1, :])
    absAc = (Ap.reshape(m, NG, L) @ Ca).reshape(m, NG * lp1)
    absBd = np.einsum("pt,gtn->gpn", Da, Bp.reshape(NG, L, -1)).reshape(NG * lp1, -1)
    return absAc, absBd


def gemm_abs_product(A, B, L, C, D, lp1):
    """sum_k |a_k| |b_k| for every output of A (m x K) times B (K x n).

    |a_k| <= sum_t |A[i, gL+t]| |C[t, p]| and |b_k| <= sum_t |D[p, t]| |B[gL+t, j]|
    over the groups g (consecutive L-chunks of K, the last zero-extended) and
    the kept projections p.  Returns (bound, number of reduced components).
    """
    A = np.abs(np.asarray(A, dtype=np.float64))
    B = np.abs(np.asarray(B, dtype=np.float64))
    m, K = A.shape
    NG = -(-K // L)
    Ap = np.zeros((m, NG * L))
    Ap[:, :K] = A
    Bp = np.zeros((NG * L, B.shape[1]))
    Bp[:K] = B
    Ca = np.abs(C[:, :lp1])
    Da = np.abs(D[:lp1, :])
    absAc = (Ap.reshape(m, NG, L) @ Ca).reshape(m, NG * lp1)
    absBd = np.einsum("pt,gtn->gpn", Da, Bp.reshape(NG, L, -1)).reshape(NG * lp1, -1)
    return absAc @ absBd, NG * lp1


def box_sums(x, w):
    """Sums of w consecutive values: out[i] = sum_{u<w} x[i+u] (valid positions)."""
    c = np.concatenate([[0.0], np.cumsum(np.asarray(x, dtype=np.float64))])
    return c[w:] - c[:-w]


def conv_abs_entries(s, k, R, mm, tt):
    """sum_g |b[m + g Lb]| |kb_t[g]| with Lb = T/R box sums of |s| and |k| (scaled by 1/Lb)."""
    T = k.shape[1]
    Lb = T // R
    bs = box_sums(np.abs(s), Lb)
    kb = np.abs(k).reshape(k.shape[0], R, Lb).sum(axis=2)
    out = np.empty(len(mm))
    for e, (m, t) in enumerate(zip(mm, tt)):
        out[e] = bs[m + Lb * np.arange(R)] @ kb[t] / Lb
    return out
