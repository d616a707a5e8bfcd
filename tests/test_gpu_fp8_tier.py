"""FP8 tier of truncated projections (pj_precision.fp8_tier) against the FP64 oracle.

The kept projections p <= l run in BF16 (plain, split, or tiered split) and the
next n projections p = l+1 .. l+n are added as an E4M3 block-scaled product
into the same FP32 output.  What is computed is the projection that keeps
l+1+n projections (Eq. 8 with l+n), so the oracle is gemm_proj at
R2 = (l+1+n) * block / L, and every output must lie within the sum of the BF16
bound of the kept components, the E4M3 bound of the tier components
(tests/helpers.py) and one FP32 rounding of the sum of the two parts.

An exactness pin fixes the bookkeeping of the tier (which basis columns it
takes, how its product is added): with the 2-point basis C = [[1, 1], [1, -1]]
and small integer inputs, every component and every partial sum is exact in
BF16, E4M3 and FP32, so keeping projection 0 in BF16 and adding projection 1 in
E4M3 must give A @ B bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
from helpers import U_BF16, U_F32, e4m3_scale_term, factor, factor_e4m3, gamma, gemm_abs_parts

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _bound(A64, B64, Kb, lp1, tier, split, kind="dct2", L=8, user_C=None):
    C, D = oracle.basis(kind, L, user_C) if user_C is not None else oracle.basis(kind, L)
    absAc, absBd = gemm_abs_parts(A64, B64, L, C, D, lp1)
    Kp = absAc.shape[1]
    kept = absAc @ absBd
    b_kept = factor(Kp * (3 if split == 2 else 1), L, split) * kept
    absAt, absBt = gemm_abs_parts(A64, B64, L, C[:, lp1:], D[lp1:, :], tier)
    tail = absAt @ absBt
    b_tier = factor_e4m3(absAt.shape[1], L, 1) * tail + e4m3_scale_term(absAt, absBt, 1)
    return b_kept + b_tier + 2 * U_F32 * (kept + tail)


@pytest.mark.parametrize("M,N,K,Kb,R,tier,split", [(300, 200, 1000, 128, 32, 6, 1), (513, 257, 777, 64, 16, 3, 1),
                                                    (129, 300, 4096, 512, 64, 7, 1), (256, 384, 2048, 256, 64, 4, 2),
                                                    (1, 1, 8, 8, 2, 3, 1), (241, 129, 136, 8, 1, 7, 2)])
def test_fp8_tier_parity_elementwise(M, N, K, Kb, R, tier, split):
    rng = np.random.default_rng(M + tier)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Y = pj.proj_gemm(At, Bt, Kb, R, split=split, fp8_tier=tier).double().cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    lp1 = R // (Kb // 8)
    ref = oracle.gemm_proj(A64, B64, Kb, (lp1 + tier) * (Kb // 8))
    bound = _bound(A64, B64, Kb, lp1, tier, split)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"


def test_fp8_tier_with_tiered_split_and_user_basis():
    """The tier after a tiered BF16 split (lo term on p = 0 only) and with an oblique
    user basis (D = C^-1 is not C^T): the tier keeps columns l+1.. of C and the same
    rows of D, so kept part plus tier is the projection onto l+1+n columns."""
    rng = np.random.default_rng(17)
    M, N, K, Kb, L = 200, 150, 640, 64, 8
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    U = np.eye(L) + 0.3 * rng.normal(size=(L, L))
    for lp1, tier, split, lead in ((2, 5, 2, 1), (3, 5, 1, 0)):
        R = lp1 * Kb // L
        Y = pj.proj_gemm(At, Bt, Kb, R, "user", L, split=split, split_lead=lead, user_C=U,
                         fp8_tier=tier).double().cpu().numpy()
        ref = oracle.gemm_proj(A64, B64, Kb, (lp1 + tier) * Kb // L, "user", L, U)
        bound = _bound(A64, B64, Kb, lp1, tier, split, "user", L, U)
        assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)


def test_fp8_tier_exact_with_two_point_basis():
    rng = np.random.default_rng(23)
    M, N, K = 160, 272, 1000
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float32)
    B = rng.integers(-8, 9, size=(K, N)).astype(np.float32)
    C = np.array([[1.0, 1.0], [1.0, -1.0]])
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Y = pj.proj_gemm(At, Bt, 100, 50, "user", 2, user_C=C, fp8_tier=1).double().cpu().numpy()
    assert np.array_equal(Y, A.astype(np.float64) @ B.astype(np.float64))
    # without the tier only projection 0 is kept: the product of the pairwise sums
    Y0 = pj.proj_gemm(At, Bt, 100, 50, "user", 2, user_C=C).double().cpu().numpy()
    assert not np.array_equal(Y0, Y)


def test_fp8_tier_staged_matches_single_call():
    rng = np.random.default_rng(29)
    M, N, K, Kb, R, tier = 384, 256, 1536, 256, 64, 4
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    Y1 = pj.proj_gemm(A, B, Kb, R, fp8_tier=tier)
    ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R, fp8_tier=tier), dtype=torch.uint8, device=DEV)
    pj.proj_gemm_project(None, B, Kb, R, ws, M=M, N=N, K=K, fp8_tier=tier)    # cached B
    pj.proj_gemm_project(A, None, Kb, R, ws, N=N, fp8_tier=tier)
    Y2 = torch.empty_like(Y1)
    pj.proj_gemm_multiply(Y2, K, Kb, R, ws, fp8_tier=tier)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)


def test_fp8_tier_rejections():
    A = torch.zeros((16, 64), device=DEV)
    B = torch.zeros((64, 16), device=DEV)
    with pytest.raises(pj.ProjError):      # l+1 + tier beyond L
        pj.proj_gemm(A, B, 64, 32, fp8_tier=5)
    with pytest.raises(pj.ProjError):      # BF16 output cannot take the added tier
        pj.proj_gemm(A, B, 64, 16, fp8_tier=2, out_dtype=torch.bfloat16)
    with pytest.raises(pj.ProjError):      # the tier is an addition to BF16 components
        pj.proj_gemm(A, B, 64, 16, compute="e4m3", fp8_tier=2)
