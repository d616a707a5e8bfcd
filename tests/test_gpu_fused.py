"""The fused project-then-multiply GEMM (proj_gemm_fused) against the FP64 oracle.

B_d is projected once into the workspace; A's groups are projected inside the
GEMM kernel (L = 8, l+1 = 8, R = block), never written to memory.  Every output
must lie within the same componentwise bound as the two-pass product
(tests/helpers.py), for plain and fully split BF16 components, FP32 and BF16
inputs, ragged M, N and K (a short last chunk of 64 samples and a last group of
fewer than 8), and the two-pass product of the same call must agree within
twice that bound.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
from helpers import factor, gemm_abs_product

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _fused(A, B, Kb, split, out_dtype=torch.float32):
    M, K = A.shape
    N = B.shape[1]
    ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, Kb, split=split), dtype=torch.uint8, device=DEV)
    pj.proj_gemm_project(None, B, Kb, Kb, ws, split=split, M=M, N=N, K=K)
    Y = torch.empty((M, N), dtype=out_dtype, device=DEV)
    pj.proj_gemm_fused(A, Y, Kb, Kb, ws, split=split)
    torch.cuda.synchronize()
    return Y


@pytest.mark.parametrize("M,N,K,Kb,split,in_dtype", [
    (300, 256, 1000, 128, 1, torch.float32),
    (513, 200, 777, 64, 2, torch.float32),      # a last group of one sample, a short last chunk (padded rows)
    (256, 512, 4096, 512, 2, torch.float32),
    (1000, 1024, 2048, 256, 1, torch.bfloat16),
    (97, 256, 520, 8, 2, torch.bfloat16),
    (4, 256, 64, 64, 1, torch.float32),         # one chunk, fewer rows than a tile
])
def test_fused_parity_elementwise(M, N, K, Kb, split, in_dtype):
    rng = np.random.default_rng(M + K)
    lda = -(-K // 8) * 8          # A's rows 16-byte aligned: a view of a wider buffer when K is not
    Abig = torch.from_numpy(rng.normal(size=(M, lda)).astype(np.float32)).to(DEV).to(in_dtype)
    A = Abig[:, :K]
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV).to(in_dtype)
    Y = _fused(A, B, Kb, split).double().cpu().numpy()
    A64, B64 = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, Kb, Kb, "dct2", 8)
    C, D = oracle.basis("dct2", 8)
    absprod, Kp = gemm_abs_product(A64, B64, 8, C, D, 8)
    bound = factor(Kp * (3 if split == 2 else 1), 8, split) * absprod
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"
    two_pass = pj.proj_gemm(A, B, Kb, Kb, split=split).double().cpu().numpy()
    assert np.all(np.abs(Y - two_pass) <= 2 * bound)


def test_fused_bf16_output_and_face_shape_sample():
    """A face-matching-shaped product (4096 probes would be the full size; 1024 here) with
    a BF16 output, against sampled oracle entries."""
    rng = np.random.default_rng(5)
    M, N, K, Kb = 1024, 2048, 10304, 512
    A = torch.from_numpy(rng.random(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    Y = _fused(A, B, Kb, 2, torch.bfloat16).double().cpu().numpy()
    ii = rng.integers(0, M, 400)
    jj = rng.integers(0, N, 400)
    A64, B64 = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = oracle.gemm_proj_entries(A64, B64, ii, jj, Kb, Kb, "dct2", 8)
    C, D = oracle.basis("dct2", 8)
    absprod, Kp = gemm_abs_product(A64[ii], B64, 8, C, D, 8)
    bound = factor(3 * Kp, 8, 2) * absprod[np.arange(400), jj]
    bound = bound + 2.0 ** -8 * (np.abs(ref) + bound)      # the BF16 output rounding
    assert np.all(np.abs(Y[ii, jj] - ref) <= bound)


def test_fused_rejections():
    A = torch.zeros((64, 256), device=DEV)
    ws = torch.empty(pj.gemm_workspace_size(64, 384, 256, 128, 64), dtype=torch.uint8, device=DEV)
    with pytest.raises(pj.ProjError):      # R < block: l+1 = 4
        pj.proj_gemm_fused(A, torch.empty((64, 384), device=DEV), 128, 64, ws)
    ws = torch.empty(pj.gemm_workspace_size(64, 384, 256, 128, 128), dtype=torch.uint8, device=DEV)
    with pytest.raises(pj.ProjError):      # three 128-row tile columns of B_d do not pair up
        pj.proj_gemm_fused(A, torch.empty((64, 384), device=DEV), 128, 128, ws)


def test_autotuned_cached_product_picks_a_measured_path(tmp_path):
    """autotune_cached_product times two_pass and fused for a cached B_d, returns the
    faster, caches the answer; proj_gemm_cached then gives the same product as the
    two-pass path within the bound (both paths are checked against it)."""
    rng = np.random.default_rng(41)
    M, N, K, Kb = 512, 512, 2048, 256
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, Kb), dtype=torch.uint8, device=DEV)
    pj.proj_gemm_project(None, B, Kb, Kb, ws, M=M, N=N, K=K)
    out = torch.empty((M, N), device=DEV)
    cache = str(tmp_path / "tune.json")
    best, trials = pj.autotune_cached_product(A, out, Kb, Kb, ws, cache=cache)
    assert best in ("two_pass", "fused")
    assert {t["path"] for t in trials} == {"two_pass", "fused"}
    assert all(t["ms"] is not None and t["ms"] > 0 for t in trials)
    assert pj.autotune_cached_product(A, out, Kb, Kb, ws, cache=cache) == (best, trials)   # from the cache
    A64, B64 = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, Kb, Kb, "dct2", 8)
    C, D = oracle.basis("dct2", 8)
    absprod, Kp = gemm_abs_product(A64, B64, 8, C, D, 8)
    bound = factor(Kp, 8, 1) * absprod
    for path in (None, "two_pass", "fused"):
        Y = pj.proj_gemm_cached(A, torch.empty_like(out), Kb, Kb, ws, path=path, cache=cache)
        torch.cuda.synchronize()
        err = np.abs(Y.double().cpu().numpy() - ref)
        assert np.all(err <= bound), (path, np.max(err / bound))
    # a shape the fused kernel refuses (R < block) is recorded and not chosen
    ws2 = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, Kb // 2), dtype=torch.uint8, device=DEV)
    pj.proj_gemm_project(None, B, Kb, Kb // 2, ws2, M=M, N=N, K=K)
    best2, trials2 = pj.autotune_cached_product(A, out, Kb, Kb // 2, ws2)
    assert best2 == "two_pass" and any(t["path"] == "fused" and t["ms"] is None for t in trials2)
