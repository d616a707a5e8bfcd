"""Pins for the FP64 oracle against things other than itself.

Each test ties an oracle function to a library routine (scipy's orthonormal
DCT-II, numpy's matmul / correlate / inverse), a textbook table, a closed
form, or a brute-force formulation with dense projection matrices built here
from those independent sources.  Together they are chosen so that a dropped
term, a wrong sign or index, a transposed operand or a mishandled tail group
in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.fft

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers ---

def dct_ortho(L):
    """Orthonormal DCT-II analysis matrix from scipy: column j = basis vector j."""
    return scipy.fft.dct(np.eye(L), type=2, norm="ortho", axis=1)


def box_projector(L, lp1):
    """Orthogonal projector onto functions constant on aligned runs of L // lp1."""
    w = L // lp1
    P = np.zeros((L, L))
    for a in range(0, L, w):
        P[a:a + w, a:a + w] = 1.0 / w
    return P


def block_projector(K, Kb, L, P_LL):
    """K x K block-diagonal operator applying the L x L map P_LL to every group.

    Blocks of Kb (last one may be short); a short last group keeps only the
    rows / columns of P_LL that exist (zero extension of the group).
    """
    Pk = np.zeros((K, K))
    for k0 in range(0, K, Kb):
        kb = min(Kb, K - k0)
        for g0 in range(0, kb, L):
            n = min(L, kb - g0)
            a = k0 + g0
            Pk[a:a + n, a:a + n] = P_LL[:n, :n]
    return Pk


def rng(seed=0):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------ basis ---

@pytest.mark.parametrize("L", [1, 2, 8, 12, 16])
def test_dct_basis_is_scipy_orthonormal_dct2(L):
    C, D = oracle.basis("dct2", L)
    np.testing.assert_allclose(C, dct_ortho(L), atol=1e-15)
    np.testing.assert_allclose(D @ C, np.eye(L), atol=1e-14)


def test_haar4_matches_textbook_table():
    ref = np.loadtxt(os.path.join(GOLDEN, "haar4.txt"))
    C, D = oracle.basis("haar", 4)
    np.testing.assert_allclose(C, ref, atol=1e-15)
    np.testing.assert_allclose(D, ref.T, atol=1e-15)


def test_haar2_is_sum_and_difference():
    C, _ = oracle.basis("haar", 2)
    np.testing.assert_allclose(C, np.array([[1, 1], [1, -1]]) / np.sqrt(2), atol=1e-15)


@pytest.mark.parametrize("L", [8, 64])
def test_haar_orthonormal_and_nested_boxes(L):
    C, D = oracle.basis("haar", L)
    np.testing.assert_allclose(C.T @ C, np.eye(L), atol=1e-14)
    lp1 = 1
    while lp1 <= L:   # first 2^j columns span the piecewise constants on L/2^j
        np.testing.assert_allclose(C[:, :lp1] @ D[:lp1, :], box_projector(L, lp1), atol=1e-14)
        lp1 *= 2


def test_user_basis_is_inverted_and_singular_rejected():
    C0 = rng(3).normal(size=(8, 8)) + 4 * np.eye(8)
    C, D = oracle.basis("user", 8, C0)
    np.testing.assert_allclose(C, C0)
    np.testing.assert_allclose(D, np.linalg.inv(C0), rtol=1e-12, atol=1e-13)
    sing = np.ones((4, 4))
    with pytest.raises(ValueError):
        oracle.basis("user", 4, sing)


# ------------------------------------------------------------------- GEMM ---

@pytest.mark.parametrize("M,K,N,Kb,L", [(7, 64, 5, 16, 8), (16, 100, 9, 32, 8), (5, 37, 3, 16, 8),
                                         (9, 48, 11, 48, 12)])
def test_gemm_full_R_equals_plain_product(M, K, N, Kb, L):
    r = rng(1)
    A, B = r.uniform(-1, 1, (M, K)), r.uniform(-1, 1, (K, N))
    Y = oracle.gemm_proj(A, B, Kb, Kb, "dct2", L)
    ref = A @ B
    assert oracle.rel_fro(Y, ref) <= 1e-14
    np.testing.assert_allclose(oracle.gemm_exact(A, B), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,L,Kb,R", [("dct2", 8, 16, 2), ("dct2", 8, 16, 6), ("dct2", 8, 32, 12),
                                          ("haar", 8, 16, 4), ("haar", 4, 8, 2), ("dct2", 4, 12, 6)])
@pytest.mark.parametrize("K", [48, 53])
def test_gemm_truncated_equals_dense_projector(kind, L, Kb, R, K):
    """Y_R = A P B with P = blockdiag(C_R C_R^T) formed from scipy's DCT or box projectors."""
    r = rng(2)
    M, N = 6, 5
    A, B = r.normal(size=(M, K)), r.normal(size=(K, N))
    lp1 = R * L // Kb
    P_LL = (dct_ortho(L)[:, :lp1] @ dct_ortho(L)[:, :lp1].T) if kind == "dct2" \
        else box_projector(L, lp1)
    Pk = block_projector(K, Kb, L, P_LL)
    np.testing.assert_allclose(oracle.gemm_proj(A, B, Kb, R, kind, L), A @ Pk @ B,
                               rtol=1e-12, atol=1e-12)


def test_gemm_closed_form_and_error_split():
    r = rng(4)
    A, B = r.normal(size=(12, 96)), r.normal(size=(96, 10))
    for R in (4, 8, 16, 32):
        YR = oracle.gemm_proj(A, B, 32, R)
        E = oracle.gemm_closed_form(A, B, 32, R)
        Y = A @ B
        assert np.linalg.norm(Y - YR - E) / np.linalg.norm(Y) <= 1e-13
        lp1 = R * 8 // 32
        P = block_projector(96, 32, 8, dct_ortho(8)[:, :lp1] @ dct_ortho(8)[:, :lp1].T)
        np.testing.assert_allclose(E, A @ (np.eye(96) - P) @ B, rtol=1e-12, atol=1e-12)


def test_gemm_oblique_user_basis():
    """Any invertible C (Eq. 5-6): the kept part is the oblique projector C_R (C^-1)_R."""
    r = rng(5)
    C0 = r.normal(size=(8, 8)) + 3 * np.eye(8)
    Ci = np.linalg.inv(C0)
    A, B = r.normal(size=(5, 40)), r.normal(size=(40, 4))
    for lp1 in (1, 3, 8):
        R = lp1 * 16 // 8
        Pk = block_projector(40, 16, 8, C0[:, :lp1] @ Ci[:lp1, :])
        np.testing.assert_allclose(oracle.gemm_proj(A, B, 16, R, "user", 8, C0), A @ Pk @ B,
                                   rtol=1e-10, atol=1e-10)
        E = oracle.gemm_closed_form(A, B, 16, R, "user", 8, C0)
        np.testing.assert_allclose(E, A @ (np.eye(40) - Pk) @ B, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("kind", ["dct2", "haar"])
def test_gemm_piecewise_constant_rows_exact_at_dc(kind):
    """Rows constant on aligned L-groups live in the DC span: l = 0 is exact (Eq. 8)."""
    r = rng(6)
    A = np.repeat(r.normal(size=(4, 6)), 8, axis=1)       # 4 x 48, constant per group
    B = r.normal(size=(48, 3))
    np.testing.assert_allclose(oracle.gemm_proj(A, B, 16, 2, kind, 8), A @ B, rtol=1e-13, atol=1e-13)


def test_gemm_L1_is_identity():
    r = rng(7)
    A, B = r.normal(size=(3, 10)), r.normal(size=(10, 4))
    np.testing.assert_allclose(oracle.gemm_proj(A, B, 5, 5, "dct2", 1), A @ B, rtol=1e-13)


def test_gemm_haar_dc_is_box_average():
    r = rng(8)
    A, B = r.normal(size=(3, 32)), r.normal(size=(32, 2))
    Abox = np.repeat(A.reshape(3, 8, 4).mean(axis=2), 4, axis=1)
    np.testing.assert_allclose(oracle.gemm_proj(A, B, 32, 8, "haar", 4), Abox @ B, rtol=1e-13)


def test_gemm_gram_parseval_and_monotone():
    """A = B^T: tr(Y - Y_R) = ||A||^2 - ||A P||^2 and the error shrinks with R."""
    r = rng(9)
    A = r.normal(size=(6, 64))
    prev = np.inf
    for R in (8, 16, 24, 32, 40, 48, 56, 64):
        E = A @ A.T - oracle.gemm_proj(A, A.T, 64, R)
        Ac = oracle.project_rows(A, 64, R)
        assert abs(np.trace(E) - (np.sum(A * A) - np.sum(Ac * Ac))) <= 1e-11
        err = np.linalg.norm(E)
        assert err <= prev + 1e-12
        prev = err
    assert prev <= 1e-12


def test_gemm_projected_shapes_printed_in_paper():
    """N = 144, L = 8, one projection: a 144 x 18 by 18 x 144 product (Sec. III-B)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_shapes.txt"))
            if l.strip() and not l.startswith("#")]
    r = rng(10)
    for kind, N, L, lp1, qty, val, *_ in rows:
        N, L, lp1 = int(N), int(L), int(lp1)
        if qty == "reduced_A_shape":
            Ac = oracle.project_rows(r.normal(size=(N, N)), N, lp1 * N // L, "dct2", L)
            assert "x".join(map(str, Ac.shape)) == val
        elif qty == "reduced_B_shape":
            Bd = oracle.project_cols(r.normal(size=(N, N)), N, lp1 * N // L, "dct2", L)
            assert "x".join(map(str, Bd.shape)) == val
        elif qty == "projected_kernel_len":
            kd = oracle.project_templates(r.normal(size=(1, N)), lp1 * N // L, "haar", L)
            assert kd.shape[1] == int(val)
        elif qty == "mac_ratio_pct":
            l = lp1 - 1
            got = 100.0 * oracle.mac_gemm_proj(N, l, L) / oracle.mac_gemm_plain(N)
            assert abs(got - float(val)) < 1e-6


def test_gemm_entries_match_full():
    r = rng(11)
    A, B = r.normal(size=(20, 70)), r.normal(size=(70, 13))
    Y = oracle.gemm_proj(A, B, 32, 12)
    ii = r.integers(0, 20, 50)
    jj = r.integers(0, 13, 50)
    np.testing.assert_allclose(oracle.gemm_proj_entries(A, B, ii, jj, 32, 12), Y[ii, jj], rtol=1e-13,
                               atol=1e-13)


def test_projected_operands_reproduce_product():
    """sum over components of A_c B_d equals Y_R (reduced products of Sec. III-B)."""
    r = rng(12)
    A, B = r.normal(size=(9, 77)), r.normal(size=(77, 6))
    Ac = oracle.project_rows(A, 32, 16)
    Bd = oracle.project_cols(B, 32, 16)
    np.testing.assert_allclose(Ac @ Bd, oracle.gemm_proj(A, B, 32, 16), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,L,user", [("dct2", 8, False), ("user", 8, True)])
def test_gemm_adjoint_matches_finite_differences(kind, L, user):
    r = rng(13)
    M, K, N, Kb, R = 4, 24, 3, 16, 4
    C0 = r.normal(size=(L, L)) + 3 * np.eye(L) if user else None
    A, B, W = r.normal(size=(M, K)), r.normal(size=(K, N)), r.normal(size=(M, N))
    dA, dB = oracle.gemm_adjoint(A, B, W, Kb, R, kind, L, C0)
    h = 1e-6

    def loss(A_, B_):
        return float(np.sum(W * oracle.gemm_proj(A_, B_, Kb, R, kind, L, C0)))

    fdA = np.zeros_like(A)
    for i in range(M):
        for k in range(K):
            Ap, Am = A.copy(), A.copy()
            Ap[i, k] += h
            Am[i, k] -= h
            fdA[i, k] = (loss(Ap, B) - loss(Am, B)) / (2 * h)
    fdB = np.zeros_like(B)
    for k in range(K):
        for j in range(N):
            Bp, Bm = B.copy(), B.copy()
            Bp[k, j] += h
            Bm[k, j] -= h
            fdB[k, j] = (loss(A, Bp) - loss(A, Bm)) / (2 * h)
    np.testing.assert_allclose(dA, fdA, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(dB, fdB, rtol=1e-7, atol=1e-8)


# ------------------------------------------------------------------- CONV ---

def test_conv_exact_is_numpy_correlate():
    r = rng(20)
    s, k = r.normal(size=300), r.normal(size=(3, 37))
    ref = np.stack([np.correlate(s, k[t], mode="valid") for t in range(3)], axis=1)
    np.testing.assert_allclose(oracle.conv_exact(s, k), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind,L", [("haar", 2), ("haar", 64), ("dct2", 8)])
def test_conv_full_R_is_exact(kind, L):
    r = rng(21)
    T = 128
    s, k = r.normal(size=700), r.normal(size=(4, T))
    ref = np.stack([np.correlate(s, k[t], mode="valid") for t in range(4)], axis=1)
    assert oracle.rel_fro(oracle.conv_proj(s, k, T, kind, L), ref) <= 1e-13


@pytest.mark.parametrize("R", [64, 32, 16, 8, 2])
def test_conv_haar_truncated_is_box_filtered_template(R):
    """Haar, l+1 = 2^j: r_R = correlation with the template box-averaged on T/R runs."""
    r = rng(22)
    T, L = 128, 64
    s, k = r.normal(size=600), r.normal(size=(3, T))
    w = T // R
    kbox = np.repeat(k.reshape(3, R, w).mean(axis=2), w, axis=1)
    ref = np.stack([np.correlate(s, kbox[t], mode="valid") for t in range(3)], axis=1)
    np.testing.assert_allclose(oracle.conv_proj(s, k, R, "haar", L), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("T,L,lp1", [(64, 8, 2), (60, 8, 2), (61, 8, 3), (61, 8, 8)])
def test_conv_dct_truncated_equals_dense_projector(T, L, lp1):
    """Includes templates whose last group is short (zero extension, Sec. III-A)."""
    r = rng(23)
    s, k = r.normal(size=250), r.normal(size=(2, T))
    C = dct_ortho(L)[:, :lp1]
    Pk = block_projector(T, T, L, C @ C.T)
    ref = np.stack([np.correlate(s, Pk @ k[t], mode="valid") for t in range(2)], axis=1)
    R = lp1 * (-(-T // L))
    np.testing.assert_allclose(oracle.conv_proj(s, k, R, "dct2", L), ref, rtol=1e-12, atol=1e-12)


def test_conv_closed_form_and_entries():
    r = rng(24)
    s, k = r.normal(size=500), r.normal(size=(5, 64))
    for R in (64, 16, 4, 1):
        rR = oracle.conv_proj(s, k, R, "haar", 64)
        e = oracle.conv_closed_form(s, k, R, "haar", 64)
        ref = oracle.conv_exact(s, k)
        assert np.linalg.norm(ref - rR - e) / np.linalg.norm(ref) <= 1e-13
        mm = r.integers(0, 500 - 64 + 1, 40)
        tt = r.integers(0, 5, 40)
        np.testing.assert_allclose(oracle.conv_proj_entries(s, k, mm, tt, R, "haar", 64), rR[mm, tt],
                                   rtol=1e-13, atol=1e-13)


def test_conv_haar_l2_dc_pairs():
    """L = 2 Haar, one projection (Sec. IV CONV setting): pairwise sums / sqrt 2 on both inputs."""
    r = rng(25)
    s, k = r.normal(size=100), r.normal(size=(1, 20))
    kd = oracle.project_templates(k, 10, "haar", 2)
    np.testing.assert_allclose(kd[0], (k[0, 0::2] + k[0, 1::2]) / np.sqrt(2), rtol=1e-14)
    rR = oracle.conv_proj(s, k, 10, "haar", 2)
    m = 7
    sc = (s[m:m + 20:2] + s[m + 1:m + 20:2]) / np.sqrt(2)
    assert abs(rR[m, 0] - sc @ kd[0]) <= 1e-12


def test_snr_definition():
    ref = np.ones(100)
    assert abs(oracle.snr_db(ref + 0.1, ref) - 20.0) < 1e-12
    assert oracle.snr_db(ref, ref) == float("inf")
    assert abs(oracle.rel_fro(ref * 1.001, ref) - 1e-3) < 1e-15


# ------------------------------------------------- interpolated lags (Sec. III-A)

def test_conv_interp_step1_and_computed_lags_are_the_projected_correlation():
    rng = np.random.default_rng(11)
    s = rng.normal(size=2500)
    k = rng.normal(size=(3, 256))
    full = oracle.conv_proj(s, k, 64)
    assert np.array_equal(oracle.conv_proj_interp(s, k, 64, 1), full)
    for step in (2, 4):
        r = oracle.conv_proj_interp(s, k, 64, step)
        assert np.array_equal(r[::step], full[::step])


def test_conv_interp_is_exact_on_affine_signals():
    """For s[n] = a + b n every correlation is affine in the lag, so interpolating
    between computed lags reproduces the projected correlation exactly."""
    n = np.arange(3001, dtype=np.float64)
    s = 0.3 - 0.002 * n
    k = np.random.default_rng(12).normal(size=(2, 256))
    full = oracle.conv_proj(s, k, 64)
    for step in (2, 4, 8):
        r = oracle.conv_proj_interp(s, k, 64, step)
        lags = full.shape[0]
        last = (lags - 1) // step * step          # lags past this one have no right neighbour
        np.testing.assert_allclose(r[:last + 1], full[:last + 1], rtol=0, atol=1e-11 * np.abs(full).max())
        assert np.array_equal(r[last + 1:], np.repeat(full[last:last + 1], lags - 1 - last, axis=0))


@pytest.mark.parametrize("step", [2, 4])
def test_conv_interp_error_within_the_linear_interpolation_bound(step):
    """A sinusoidal signal gives a sinusoidal correlation r[m] = A cos(w m + psi);
    linear interpolation over h = step lags errs by at most h^2 w^2 A / 8."""
    w = 2 * np.pi / 97.0
    n = np.arange(4000, dtype=np.float64)
    s = np.cos(w * n + 0.4)
    k = np.random.default_rng(13).normal(size=(2, 512))
    full = oracle.conv_proj(s, k, 128)
    r = oracle.conv_proj_interp(s, k, 128, step)
    m = np.arange(full.shape[0], dtype=np.float64)
    basis = np.stack([np.cos(w * m), np.sin(w * m)], axis=1)
    coef, *_ = np.linalg.lstsq(basis, full, rcond=None)
    amp = np.sqrt((coef ** 2).sum(axis=0))                    # A per template
    assert np.allclose(basis @ coef, full, atol=1e-9 * amp.max())   # it is a sinusoid
    lags = full.shape[0]
    last = (lags - 1) // step * step
    err = np.abs(r[:last + 1] - full[:last + 1])
    bound = step ** 2 * w ** 2 * amp / 8
    assert np.all(err <= bound * (1 + 1e-9) + 1e-12), (err.max(axis=0), bound)
    assert err.max() > 0.1 * bound.min()                      # and the interpolation is used


def test_conv_interp_entries_match_full():
    rng = np.random.default_rng(14)
    s = rng.normal(size=1999)
    k = rng.normal(size=(2, 128))
    r = oracle.conv_proj_interp(s, k, 32, 2)
    mm = np.concatenate([rng.integers(0, r.shape[0], 200), [r.shape[0] - 1, r.shape[0] - 2, 0]])
    tt = rng.integers(0, 2, len(mm))
    np.testing.assert_allclose(oracle.conv_proj_interp_entries(s, k, mm, tt, 32, 2), r[mm, tt], rtol=1e-13,
                               atol=1e-13)


# ---------------------------------------------- learned (PCA) basis (Sec. V-A) --

def pca_group_basis(A, L):
    """Principal axes of the L-sample groups of A's rows, largest variance first
    (the learned basis of the face-recognition application), as the columns of C."""
    G = np.asarray(A, dtype=np.float64).reshape(-1, L)
    w, V = np.linalg.eigh(G.T @ G / G.shape[0])
    return V[:, ::-1].copy()


def test_pca_basis_beats_dct_on_its_own_data():
    """A basis learned from A keeps more of A's energy than the DCT at every l+1
    (Eckart-Young on the groups), and with an isotropic B the projected product
    errs less too."""
    from synth import face_probes
    A = face_probes(64, seed=3).astype(np.float64)
    B = np.random.default_rng(4).normal(size=(A.shape[1], 48))
    L, Kb = 8, 512
    C = pca_group_basis(A, L)
    ex = A @ B
    for lp1 in (1, 2, 4):
        R = lp1 * Kb // L
        kept_pca = oracle.project_rows(A, Kb, R, "user", L, C)
        kept_dct = oracle.project_rows(A, Kb, R, "dct2", L)
        assert np.sum(kept_pca ** 2) >= np.sum(kept_dct ** 2) * (1 - 1e-12)
        e_pca = oracle.rel_fro(oracle.gemm_proj(A, B, Kb, R, "user", L, C), ex)
        e_dct = oracle.rel_fro(oracle.gemm_proj(A, B, Kb, R, "dct2", L), ex)
        assert e_pca <= e_dct * 1.02, (lp1, e_pca, e_dct)
