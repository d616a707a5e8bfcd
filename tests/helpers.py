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
