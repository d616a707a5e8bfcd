"""proj_gemm_report: the a-posteriori truncation and rounding bounds against the
FP64 oracle and against a direct computation of the per-block residuals."""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _residual_norms(X, Kb, L, lp1, C, D, rows):
    """||X_b (I - P_b)||_F per inner block b (rows=True: blocks of columns of A;
    rows=False: blocks of rows of B), from explicit residuals in FP64."""
    out = []
    K = X.shape[1] if rows else X.shape[0]
    for k0 in range(0, K, Kb):
        k1 = min(K, k0 + Kb)
        Xb = X[:, k0:k1] if rows else X[k0:k1, :].T
        n = -(-(k1 - k0) // L) * L
        Xp = np.zeros((Xb.shape[0], n))
        Xp[:, :k1 - k0] = Xb
        G = Xp.reshape(Xb.shape[0], -1, L)
        if rows:
            kept = (G @ C[:, :lp1]) @ D[:lp1, :]
        else:
            kept = (G @ D[:lp1, :].T) @ C[:, :lp1].T
        out.append(np.linalg.norm(G - kept))
    return np.array(out)


@pytest.mark.parametrize("compute,split,R", [("bf16", 1, 32), ("bf16", 2, 64), ("f64", 1, 32), ("bf16", 1, 128)])
def test_report_bounds_hold_and_match(compute, split, R):
    rng = np.random.default_rng(3)
    M, N, K, Kb, L = 300, 200, 1000, 128, 8
    lp1 = R // (Kb // L)
    A = rng.normal(size=(M, K)).cumsum(axis=1) / 10   # smooth rows: most energy in the low projections
    B = rng.normal(size=(K, N))
    dt = torch.float64 if compute == "f64" else torch.float32
    At, Bt = torch.from_numpy(A).to("cuda", dt), torch.from_numpy(B).to("cuda", dt)
    A64, B64 = At.double().cpu().numpy(), Bt.double().cpu().numpy()
    rep = pj.proj_gemm_report(At, Bt, Kb, R, compute=compute, split=split)
    C, D = oracle.basis("dct2", L)
    expect = float(np.sum(_residual_norms(A64, Kb, L, lp1, C, D, True) * _residual_norms(B64, Kb, L, lp1, C, D, False)))
    assert abs(rep["trunc_bound"] - expect) <= 1e-9 * max(expect, 1e-300) + 1e-9 * np.linalg.norm(A64) * np.linalg.norm(B64)
    Y_R = oracle.gemm_proj(A64, B64, Kb, R, "dct2", L)
    assert np.linalg.norm(A64 @ B64 - Y_R) <= rep["trunc_bound"] * (1 + 1e-9) + 1e-9
    Y = pj.proj_gemm(At, Bt, Kb, R, compute=compute, split=split).double().cpu().numpy()
    assert np.linalg.norm(Y - Y_R) <= rep["round_bound"]
    assert abs(rep["norm_A"] - np.linalg.norm(A64)) <= 1e-10 * np.linalg.norm(A64)
    assert abs(rep["norm_B"] - np.linalg.norm(B64)) <= 1e-10 * np.linalg.norm(B64)
    nb = -(-K // Kb)
    Kp = (nb - 1) * R + lp1 * -(-(K - (nb - 1) * Kb) // L)
    passes = 3 if split == 2 else 1
    assert rep["alg_flops"] == 2.0 * M * N * Kp * passes + 2.0 * (M + N) * K * lp1
    es = 8 if compute == "f64" else 4
    assert rep["alg_bytes"] == es * (M * K + K * N) + es * M * N
    if R == Kb:
        assert rep["trunc_bound"] <= 1e-6 * np.linalg.norm(A64) * np.linalg.norm(B64)


def test_report_user_basis_and_e4m3_mark_missing_bounds():
    rng = np.random.default_rng(4)
    A = torch.from_numpy(rng.normal(size=(64, 256)).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.normal(size=(256, 64)).astype(np.float32)).cuda()
    uc = rng.normal(size=(8, 8)) + 3 * np.eye(8)
    rep = pj.proj_gemm_report(A, B, 64, 16, basis="user", user_C=uc)
    assert rep["trunc_bound"] == -1.0 and rep["round_bound"] > 0
    rep = pj.proj_gemm_report(A, B, 64, 16, compute="e4m3", split=2)
    assert rep["round_bound"] == -1.0 and rep["trunc_bound"] >= 0
