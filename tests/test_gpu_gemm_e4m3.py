"""Projected GEMM with FP8 (E4M3) block-scaled components against the FP64 oracle.

The components are quantised per run of 32 reduced components with a
power-of-two scale, and the reduced product runs on the block-scaled tcgen05
MMA.  Parity is checked elementwise against the bound of tests/helpers.py
(E4M3 part), and one exactness test pins the scale bookkeeping: with L = 1
(the identity projection) and inputs whose values E4M3 represents exactly
after any power-of-two scaling, the product must equal A @ B exactly.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
from helpers import e4m3_scale_term, factor_e4m3, gemm_abs_parts

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _e4m3_case(M, N, K, Kb, R, split, kind="dct2", L=8, in_dtype=torch.float32, out_dtype=torch.float32, seed=2):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    At = torch.from_numpy(A).to(DEV).to(in_dtype)
    Bt = torch.from_numpy(B).to(DEV).to(in_dtype)
    A64 = At.double().cpu().numpy()
    B64 = Bt.double().cpu().numpy()
    Y = pj.proj_gemm(At, Bt, Kb, R, kind, L, compute="e4m3", split=split, out_dtype=out_dtype)
    Y = Y.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, Kb, R, kind, L)
    C, D = oracle.basis(kind, L)
    lp1 = R // (Kb // L)
    absAc, absBd = gemm_abs_parts(A64, B64, L, C, D, lp1)
    Kp = absAc.shape[1]
    bound = factor_e4m3(Kp * (3 if split == 2 else 1), L, split) * (absAc @ absBd) + \
        e4m3_scale_term(absAc, absBd, split)
    if out_dtype == torch.bfloat16:
        bound += 2.0 ** -8 * (np.abs(ref) + bound)
    return Y, ref, bound


@pytest.mark.parametrize("M,N,K,Kb,R", [(300, 200, 1000, 128, 32), (256, 128, 512, 128, 128),
                                         (513, 257, 777, 64, 16), (1, 1, 8, 8, 8), (129, 300, 4096, 512, 64),
                                         (640, 384, 2048, 256, 256), (241, 129, 136, 8, 8)])
@pytest.mark.parametrize("split", [1, 2])
def test_e4m3_parity_elementwise(M, N, K, Kb, R, split):
    Y, ref, bound = _e4m3_case(M, N, K, Kb, R, split)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"
    if M * N >= 1000:  # a norm-wise check needs many outputs; a single short dot product may cancel
        rel = oracle.rel_fro(Y, ref)
        assert rel <= (0.1 if split == 1 else 5e-3), rel


def _exact_operands(M, N, K, seed):
    """Integers in [-8, 8] (exact in E4M3) times powers of two: per row of A,
    per column of B, and per 32-run of K with opposite signs of the exponent
    on the two sides, so every block scale differs but every product is exact."""
    rng = np.random.default_rng(seed)
    h = rng.integers(-10, 11, size=-(-K // 32)).repeat(32)[:K]
    ea = rng.integers(-12, 13, size=M)
    fb = rng.integers(-12, 13, size=N)
    A = rng.integers(-8, 9, size=(M, K)) * np.exp2(ea[:, None] + h[None, :])
    B = rng.integers(-8, 9, size=(K, N)) * np.exp2(fb[None, :] - h[:, None])
    return A.astype(np.float32), B.astype(np.float32)


@pytest.mark.parametrize("M,N,K", [(250, 130, 512), (37, 300, 1000), (480, 256, 4096)])
@pytest.mark.parametrize("split", [1, 2])
def test_e4m3_exact_with_identity_projection(M, N, K, split):
    A, B = _exact_operands(M, N, K, seed=M + K)
    Y = pj.proj_gemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), 64, 64, "dct2", 1,
                     compute="e4m3", split=split).double().cpu().numpy()
    ex = A.astype(np.float64) @ B.astype(np.float64)
    assert np.array_equal(Y, ex), np.max(np.abs(Y - ex))


def test_e4m3_stream_k_schedule():
    """6 tiles of 471 K stages: stream-K over all SMs with partial products added."""
    Y, ref, bound = _e4m3_case(300, 260, 20000, 128, 128, 2, seed=9)
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)
    assert oracle.rel_fro(Y, ref) <= 5e-3


def test_e4m3_bf16_inputs_and_outputs():
    Y, ref, bound = _e4m3_case(300, 260, 640, 128, 64, 2, in_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    assert np.all(np.abs(Y - ref) <= bound)


@pytest.mark.parametrize("kind,L,Kb,R", [("haar", 8, 64, 16), ("dct2", 16, 128, 48)])
def test_e4m3_other_bases(kind, L, Kb, R):
    Y, ref, bound = _e4m3_case(200, 150, 333, Kb, R, 2, kind, L)
    assert np.all(np.abs(Y - ref) <= bound)


def test_e4m3_full_R_against_exact_product():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(512, 1024)).astype(np.float32)
    B = rng.normal(size=(1024, 256)).astype(np.float32)
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    ex = A.astype(np.float64) @ B.astype(np.float64)
    y1 = pj.proj_gemm(At, Bt, 128, 128, compute="e4m3", split=1).double().cpu().numpy()
    y2 = pj.proj_gemm(At, Bt, 128, 128, compute="e4m3", split=2).double().cpu().numpy()
    assert oracle.rel_fro(y1, ex) <= 0.1
    assert oracle.rel_fro(y2, ex) <= 5e-3
    assert oracle.rel_fro(y2, ex) < oracle.rel_fro(y1, ex) / 8


def test_e4m3_staged_project_then_multiply_matches_single_call():
    rng = np.random.default_rng(4)
    A = torch.from_numpy(rng.normal(size=(300, 512)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(512, 200)).astype(np.float32)).to(DEV)
    Y1 = pj.proj_gemm(A, B, 128, 32, compute="e4m3", split=2)
    ws = torch.empty(pj.gemm_workspace_size(300, 200, 512, 128, 32, compute="e4m3", split=2), dtype=torch.uint8,
                     device=DEV)
    pj.proj_gemm_project(A, B, 128, 32, ws, compute="e4m3", split=2)
    Y2 = torch.empty((300, 200), device=DEV)
    pj.proj_gemm_multiply(Y2, 512, 128, 32, ws, compute="e4m3", split=2)
    pj.check(ws)
    assert torch.equal(Y1, Y2)


def test_e4m3_backward_is_rejected():
    A = torch.zeros((8, 64), device=DEV)
    B = torch.zeros((64, 8), device=DEV)
    with pytest.raises(pj.ProjError):
        pj.proj_gemm_backward(A, B, torch.zeros((8, 8), device=DEV), 64, 16, compute="e4m3")


@pytest.mark.parametrize("M,N,K", [(250, 300, 1000), (480, 256, 4096), (64, 264, 520)])
@pytest.mark.parametrize("split", [1, 2])
def test_e4m3_written_by_the_projection_is_exact_with_identity_basis(M, N, K, split):
    """The projection kernel writes E4M3 components and block scales itself where the
    rows suit TMA (L = 8, l+1 = 8 on both sides here).  With C = I (a user basis) the
    components are the inputs in their own order, so the exact operands of the L = 1
    pin must again give A @ B exactly: the runs, scales, padding and tails of the
    projection's E4M3 output are those the block-scaled MMA reads."""
    A, B = _exact_operands(M, N, K, seed=M + 7 * K)
    Y = pj.proj_gemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), 64, 64, "user", 8,
                     user_C=np.eye(8), compute="e4m3", split=split).double().cpu().numpy()
    ex = A.astype(np.float64) @ B.astype(np.float64)
    assert np.array_equal(Y, ex), np.max(np.abs(Y - ex))


@pytest.mark.parametrize("R", [8, 16, 32, 64])
def test_e4m3_projection_written_rows_match_the_quantiser_pass(R):
    """A's rows projected straight to E4M3 (16-byte row pitch; A projected alone, B_d
    cached, so the projection takes A by itself) and through the BF16 pairs and the
    quantiser pass (a view whose pitch is not a 16-byte multiple): both products lie
    within the E4M3 bound of the oracle and within twice it of each other."""
    rng = np.random.default_rng(R)
    M, N, K, Kb = 300, 264, 1024, 64
    Abig = rng.normal(size=(M, K + 1)).astype(np.float32)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    A_al = torch.from_numpy(np.ascontiguousarray(Abig[:, :K])).to(DEV)
    A_un = torch.from_numpy(Abig).to(DEV)[:, :K]
    Ys = []
    for A_ in (A_al, A_un):
        ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R, compute="e4m3", split=2), dtype=torch.uint8,
                         device=DEV)
        pj.proj_gemm_project(None, B, Kb, R, ws, compute="e4m3", split=2, M=M, N=N, K=K)
        pj.proj_gemm_project(A_, None, Kb, R, ws, compute="e4m3", split=2, N=N)
        Y = torch.empty((M, N), device=DEV)
        pj.proj_gemm_multiply(Y, K, Kb, R, ws, compute="e4m3", split=2)
        pj.check(ws)
        Ys.append(Y.double().cpu().numpy())
    A64, B64 = Abig[:, :K].astype(np.float64), B.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, Kb, R)
    C, D = oracle.basis("dct2", 8)
    lp1 = R // (Kb // 8)
    absAc, absBd = gemm_abs_parts(A64, B64, 8, C, D, lp1)
    bound = factor_e4m3(absAc.shape[1] * 3, 8, 2) * (absAc @ absBd) + e4m3_scale_term(absAc, absBd, 2)
    for Y in Ys:
        assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)
    assert np.all(np.abs(Ys[0] - Ys[1]) <= 2 * bound)
