"""FP64 CPU oracle for projected GEMM / CONV (arXiv 1411.2860).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1411_2860_gb300`` and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
independent output rows); this module compiles it with gcc on first use and
wraps it with numpy.  Every function cites the passage of the paper it
follows (section / equation numbers of the TCSVT 2014 paper).

Parity status: every public function here is pinned by ``tests/test_oracle_pins.py``
(library routines, closed forms, brute force on tiny inputs, special cases).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BASIS = {"dct2": 0, "haar": 1, "user": 2}

_d = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_threads.argtypes = [_int]
            lib.or_threads.restype = _int
            lib.or_basis.argtypes = [_int, _int, _d, _d, _d]
            lib.or_basis.restype = _int
            lib.or_gemm_exact.argtypes = [_d, _d, _d, _i64, _i64, _i64, _int]
            lib.or_gemm_proj.argtypes = [_d, _d, _d, _i64, _i64, _i64, _i64, _int, _int, _d, _d, _int]
            lib.or_gemm_closed_form.argtypes = [_d, _d, _d, _i64, _i64, _i64, _i64, _int, _int, _d, _d, _int]
            lib.or_gemm_closed_form.restype = _int
            lib.or_gemm_adjoint.argtypes = [_d, _d, _d, _d, _d, _i64, _i64, _i64, _i64, _int, _int, _d, _d, _int]
            lib.or_gemm_proj_entries.argtypes = [_d, _d, _i64, _i64, _i64, _i64, _int, _int, _d, _d,
                                                 _i64p, _i64p, _i64, _d, _int]
            lib.or_conv_exact.argtypes = [_d, _i64, _d, _i64, _i64, _d, _int]
            lib.or_conv_proj.argtypes = [_d, _i64, _d, _i64, _i64, _int, _int, _d, _d, _d, _int]
            lib.or_conv_proj.restype = _int
            lib.or_conv_proj_entries.argtypes = [_d, _i64, _d, _i64, _i64, _int, _int, _d, _d,
                                                 _i64p, _i64p, _i64, _d, _int]
            lib.or_conv_proj_entries.restype = _int
            lib.or_conv_proj_interp.argtypes = [_d, _i64, _d, _i64, _i64, _int, _int, _d, _d, _i64, _d, _int]
            lib.or_conv_proj_interp.restype = _int
            lib.or_conv_closed_form.argtypes = [_d, _i64, _d, _i64, _i64, _int, _int, _d, _d, _d, _int]
            lib.or_conv_closed_form.restype = _int
            lib.or_project_rows.argtypes = [_d, _i64, _i64, _i64, _int, _int, _d, _d]
            lib.or_project_rows.restype = _i64
            lib.or_project_cols.argtypes = [_d, _i64, _i64, _i64, _int, _int, _d, _d]
            lib.or_project_cols.restype = _i64
            lib.or_project_templates.argtypes = [_d, _i64, _i64, _int, _int, _d, _d]
            lib.or_project_templates.restype = _i64
            _lib = lib
    return _lib


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(x: np.ndarray):
    return x.ctypes.data_as(_d)


def threads(nthreads: int = 0) -> int:
    """Threads an oracle call with ``nthreads`` (0 = OpenMP default) runs on."""
    return int(_load().or_threads(int(nthreads)))


def basis(kind: str = "dct2", L: int = 8, user_C=None):
    """Projection pair (C, D = C^-1), Eq. 5-7.

    C[i, j] = c[i, j]; column j is projection vector j.  DCT-II (Eq. 7) and Haar
    columns are scaled to unit length so D = C^T; a user matrix is inverted
    (Gauss-Jordan, partial pivoting).
    """
    lib = _load()
    C = np.zeros((L, L))
    D = np.zeros((L, L))
    uc = _f64(user_C) if user_C is not None else None
    rc = lib.or_basis(BASIS[kind], int(L), _p(uc) if uc is not None else None, _p(C), _p(D))
    if rc != 0:
        raise ValueError(f"oracle basis: invalid ({kind}, L={L}) or singular matrix")
    return C, D


def _lp1(R: int, block: int, L: int) -> int:
    """l+1 from R = (l+1) * ceil(block / L): R components kept per block of `block`.

    A block whose length is not a multiple of L has a zero-extended last group.
    """
    G = -(-block // L)
    if R % G:
        raise ValueError(f"R={R} is not (l+1)*ceil(block/L) for block={block}, L={L}")
    lp1 = R // G
    if not 1 <= lp1 <= L:
        raise ValueError(f"R={R} gives l+1={lp1} outside [1, L={L}]")
    return lp1


def gemm_exact(A, B, nthreads: int = 0) -> np.ndarray:
    """Y = A B (Eq. 2)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Y = np.empty((M, N))
    _load().or_gemm_exact(_p(A), _p(B), _p(Y), M, N, K, nthreads)
    return Y


def gemm_proj(A, B, block_k: int, R: int, kind: str = "dct2", L: int = 8, user_C=None,
              nthreads: int = 0) -> np.ndarray:
    """Projected GEMM keeping R = (l+1) block_k / L components per block (Sec. III-B)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    N = B.shape[1]
    lp1 = _lp1(R, block_k, L)
    C, D = basis(kind, L, user_C)
    Y = np.empty((M, N))
    _load().or_gemm_proj(_p(A), _p(B), _p(Y), M, N, K, block_k, L, lp1, _p(C), _p(D), nthreads)
    return Y


def gemm_closed_form(A, B, block_k: int, R: int, kind: str = "dct2", L: int = 8, user_C=None,
                     nthreads: int = 0) -> np.ndarray:
    """E = Y - Y_R = A (I - P) B with P = blockdiag(C_R D_R)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    N = B.shape[1]
    lp1 = _lp1(R, block_k, L)
    C, D = basis(kind, L, user_C)
    E = np.empty((M, N))
    rc = _load().or_gemm_closed_form(_p(A), _p(B), _p(E), M, N, K, block_k, L, lp1, _p(C), _p(D), nthreads)
    if rc:
        raise RuntimeError("oracle closed form failed")
    return E


def gemm_adjoint(A, B, dY, block_k: int, R: int, kind: str = "dct2", L: int = 8, user_C=None,
                 nthreads: int = 0):
    """(dA, dB) of sum(dY * Y_R): dA = dY B^T P^T, dB = P^T A^T dY (dense P per block)."""
    A, B, dY = _f64(A), _f64(B), _f64(dY)
    M, K = A.shape
    N = B.shape[1]
    lp1 = _lp1(R, block_k, L)
    C, D = basis(kind, L, user_C)
    dA = np.empty((M, K))
    dB = np.empty((K, N))
    _load().or_gemm_adjoint(_p(A), _p(B), _p(dY), _p(dA), _p(dB), M, N, K, block_k, L, lp1,
                            _p(C), _p(D), nthreads)
    return dA, dB


def gemm_proj_entries(A, B, ii, jj, block_k: int, R: int, kind: str = "dct2", L: int = 8,
                      user_C=None, nthreads: int = 0) -> np.ndarray:
    """Y_R[ii[e], jj[e]] for each e, by the same steps as gemm_proj."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    N = B.shape[1]
    lp1 = _lp1(R, block_k, L)
    C, D = basis(kind, L, user_C)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.empty(len(ii))
    _load().or_gemm_proj_entries(_p(A), _p(B), M, N, K, block_k, L, lp1, _p(C), _p(D),
                                 ii.ctypes.data_as(_i64p), jj.ctypes.data_as(_i64p), len(ii),
                                 _p(out), nthreads)
    return out


def conv_exact(s, k, nthreads: int = 0) -> np.ndarray:
    """Valid cross-correlation r[m, t] = sum_n s[m+n] k[t, n] (Sec. II-B, Eq. 3 with k[m+n])."""
    s = _f64(s)
    k = _f64(np.atleast_2d(k))
    nt, T = k.shape
    S = s.shape[0]
    r = np.empty((S - T + 1, nt))
    _load().or_conv_exact(_p(s), S, _p(k), T, nt, _p(r), nthreads)
    return r


def conv_proj(s, k, R: int, kind: str = "haar", L: int = 64, user_C=None,
              nthreads: int = 0) -> np.ndarray:
    """Projected valid cross-correlation, all lags (Eq. 11-13, zero-extended translations).

    The block is the template length T; R = (l+1) T / L components are kept.
    """
    s = _f64(s)
    k = _f64(np.atleast_2d(k))
    nt, T = k.shape
    S = s.shape[0]
    lp1 = _lp1(R, T, L)
    C, D = basis(kind, L, user_C)
    r = np.empty((S - T + 1, nt))
    rc = _load().or_conv_proj(_p(s), S, _p(k), T, nt, L, lp1, _p(C), _p(D), _p(r), nthreads)
    if rc:
        raise RuntimeError("oracle conv_proj failed")
    return r


def conv_proj_entries(s, k, mm, tt, R: int, kind: str = "haar", L: int = 64, user_C=None,
                      nthreads: int = 0) -> np.ndarray:
    """r_R[mm[e], tt[e]] for each e, by the same steps as conv_proj."""
    s = _f64(s)
    k = _f64(np.atleast_2d(k))
    nt, T = k.shape
    S = s.shape[0]
    lp1 = _lp1(R, T, L)
    C, D = basis(kind, L, user_C)
    mm = np.ascontiguousarray(mm, dtype=np.int64)
    tt = np.ascontiguousarray(tt, dtype=np.int64)
    out = np.empty(len(mm))
    rc = _load().or_conv_proj_entries(_p(s), S, _p(k), T, nt, L, lp1, _p(C), _p(D),
                                      mm.ctypes.data_as(_i64p), tt.ctypes.data_as(_i64p), len(mm),
                                      _p(out), nthreads)
    if rc:
        raise RuntimeError("oracle conv_proj_entries failed")
    return out


def conv_proj_interp(s, k, R: int, step: int, kind: str = "haar", L: int = 64, user_C=None,
                     nthreads: int = 0) -> np.ndarray:
    """Projected correlation computed at every step-th lag, the lags between filled by
    linear interpolation of their two computed neighbours (Sec. III-A; step = 2 is the
    half-sample option: average of the two neighbours).  A lag past the last computed
    one keeps the nearest computed value."""
    s = _f64(s)
    k = _f64(np.atleast_2d(k))
    nt, T = k.shape
    S = s.shape[0]
    lp1 = _lp1(R, T, L)
    C, D = basis(kind, L, user_C)
    r = np.empty((S - T + 1, nt))
    rc = _load().or_conv_proj_interp(_p(s), S, _p(k), T, nt, L, lp1, _p(C), _p(D), int(step), _p(r), nthreads)
    if rc:
        raise RuntimeError("oracle conv_proj_interp failed")
    return r


def conv_proj_interp_entries(s, k, mm, tt, R: int, step: int, kind: str = "haar", L: int = 64, user_C=None,
                             nthreads: int = 0) -> np.ndarray:
    """conv_proj_interp at selected (lag, template) entries: the computed neighbours
    come from conv_proj_entries and are combined as conv_proj_interp combines them."""
    mm = np.asarray(mm, dtype=np.int64)
    tt = np.asarray(tt, dtype=np.int64)
    lags = np.asarray(s).shape[0] - np.atleast_2d(k).shape[1] + 1
    m0 = mm - mm % step
    m1 = m0 + step
    has1 = m1 < lags
    r0 = conv_proj_entries(s, k, m0, tt, R, kind, L, user_C, nthreads)
    r1 = conv_proj_entries(s, k, np.where(has1, m1, m0), tt, R, kind, L, user_C, nthreads)
    out = np.where(has1, ((m1 - mm) * r0 + (mm - m0) * r1) / step, r0)
    return np.where(mm == m0, r0, out)


def conv_closed_form(s, k, R: int, kind: str = "haar", L: int = 64, user_C=None,
                     nthreads: int = 0) -> np.ndarray:
    """e = r - r_R = <s[m .. m+T), (I - P) k_t>."""
    s = _f64(s)
    k = _f64(np.atleast_2d(k))
    nt, T = k.shape
    S = s.shape[0]
    lp1 = _lp1(R, T, L)
    C, D = basis(kind, L, user_C)
    e = np.empty((S - T + 1, nt))
    rc = _load().or_conv_closed_form(_p(s), S, _p(k), T, nt, L, lp1, _p(C), _p(D), _p(e), nthreads)
    if rc:
        raise RuntimeError("oracle conv closed form failed")
    return e


def project_rows(A, block_k: int, R: int, kind: str = "dct2", L: int = 8, user_C=None):
    """A_c: every row of A projected group by group (Sec. III-B, Fig. 5 left half).

    Columns are ordered block by block, then group g, then projection p.
    """
    A = _f64(A)
    M, K = A.shape
    lp1 = _lp1(R, block_k, L)
    C, _ = basis(kind, L, user_C)
    lib = _load()
    w = lib.or_project_rows(_p(A), M, K, block_k, L, lp1, _p(C), None)
    out = np.empty((M, w))
    lib.or_project_rows(_p(A), M, K, block_k, L, lp1, _p(C), _p(out))
    return out


def project_cols(B, block_k: int, R: int, kind: str = "dct2", L: int = 8, user_C=None):
    """B_d: every column of B projected group by group (Sec. III-B, Fig. 5 right half)."""
    B = _f64(B)
    K, N = B.shape
    lp1 = _lp1(R, block_k, L)
    _, D = basis(kind, L, user_C)
    lib = _load()
    h = lib.or_project_cols(_p(B), K, N, block_k, L, lp1, _p(D), None)
    out = np.empty((h, N))
    lib.or_project_cols(_p(B), K, N, block_k, L, lp1, _p(D), _p(out))
    return out


def project_templates(k, R: int, kind: str = "haar", L: int = 64, user_C=None):
    """k_d: templates projected group by group (Eq. 12 per group, Fig. 6 bottom half)."""
    k = _f64(np.atleast_2d(k))
    nt, T = k.shape
    lp1 = _lp1(R, T, L)
    _, D = basis(kind, L, user_C)
    lib = _load()
    w = lib.or_project_templates(_p(k), T, nt, L, lp1, _p(D), None)
    out = np.empty((nt, w))
    lib.or_project_templates(_p(k), T, nt, L, lp1, _p(D), _p(out))
    return out


def rel_fro(x, ref) -> float:
    """Relative Frobenius error ||x - ref||_F / ||ref||_F."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / den) if den > 0 else float(np.linalg.norm(x - ref))


def snr_db(x, ref) -> float:
    """SNR of Eq. 9: 10 log10(sum r^2 / sum (r - r_hat)^2)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = float(np.sum(ref * ref))
    den = float(np.sum((ref - x) ** 2))
    return float("inf") if den == 0 else 10.0 * np.log10(num / den)


def mac_gemm_plain(N: int) -> int:
    """MACs of a plain N x N by N x N subblock product (Eq. 16)."""
    return N ** 3


def mac_gemm_proj(N: int, l: int, L: int) -> float:
    """MACs of the projected subblock product with l+1 of L projections (Eq. 17)."""
    return N * N * ((l + 1) / L * N + 3 * l + 2)
