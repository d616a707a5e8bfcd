"""Gradients of the projected GEMM: FP64 against finite differences, torch.gradcheck and
the oracle's adjoint; BF16 against the oracle's adjoint within a derived bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
import synth
from helpers import U_BF16, gamma

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def test_f64_gradcheck_64x128x64():
    """Finite-difference check in FP64 at 64 x 128 x 64, block 128, R = 32 (l+1 = 2, L = 8)."""
    rng = np.random.default_rng(0)
    A = torch.from_numpy(rng.normal(size=(64, 128))).to(DEV).requires_grad_()
    B = torch.from_numpy(rng.normal(size=(128, 64))).to(DEV).requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b: pj.proj_matmul(a, b, 128, 32), (A, B), eps=1e-6, atol=1e-8,
                                    rtol=1e-6)


@pytest.mark.parametrize("kind,L,Kb,R,K", [("dct2", 8, 128, 32, 128), ("haar", 8, 64, 16, 200),
                                            ("user", 8, 32, 12, 77), ("dct2", 8, 64, 64, 130)])
def test_f64_adjoint_matches_oracle(kind, L, Kb, R, K):
    rng = np.random.default_rng(1)
    M, N = 48, 40
    A, B, W = rng.normal(size=(M, K)), rng.normal(size=(K, N)), rng.normal(size=(M, N))
    uc = rng.normal(size=(L, L)) + 3 * np.eye(L) if kind == "user" else None
    dA, dB = pj.proj_gemm_backward(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV),
                                   torch.from_numpy(W).to(DEV), Kb, R, kind, L, user_C=uc)
    rA, rB = oracle.gemm_adjoint(A, B, W, Kb, R, kind, L, uc)
    assert oracle.rel_fro(dA.cpu().numpy(), rA) <= 1e-12
    assert oracle.rel_fro(dB.cpu().numpy(), rB) <= 1e-12


def test_f64_finite_differences_small():
    """Central differences of sum(W * Y_R) against the adjoint, entry by entry."""
    rng = np.random.default_rng(2)
    A, B, W = rng.normal(size=(6, 32)), rng.normal(size=(32, 5)), rng.normal(size=(6, 5))
    At, Bt, Wt = (torch.from_numpy(x).to(DEV) for x in (A, B, W))
    dA, dB = pj.proj_gemm_backward(At, Bt, Wt, 16, 4)
    h = 1e-6

    def loss(a, b):
        return float((pj.proj_gemm(a, b, 16, 4) * Wt).sum())

    for (i, k) in [(0, 0), (3, 17), (5, 31)]:
        Ap, Am = At.clone(), At.clone()
        Ap[i, k] += h
        Am[i, k] -= h
        assert abs((loss(Ap, Bt) - loss(Am, Bt)) / (2 * h) - float(dA[i, k])) <= 1e-7 * (1 + abs(float(dA[i, k])))
    for (k, j) in [(0, 0), (20, 3), (31, 4)]:
        Bp, Bm = Bt.clone(), Bt.clone()
        Bp[k, j] += h
        Bm[k, j] -= h
        assert abs((loss(At, Bp) - loss(At, Bm)) / (2 * h) - float(dB[k, j])) <= 1e-7 * (1 + abs(float(dB[k, j])))


def _bf16_grad_bounds(A, B, W, Kb, R, L, rows, cols):
    """Elementwise bounds for dA[rows] and dB[:, cols] of the BF16 path (see helpers)."""
    C, D = oracle.basis("dct2", L)
    lp1 = R // (Kb // L)
    K = A.shape[1]
    NG = -(-K // L)
    pad = NG * L - K
    Ca, Da = np.abs(C[:, :lp1]), np.abs(D[:lp1, :])
    absA = np.pad(np.abs(A), ((0, 0), (0, pad)))
    absB = np.pad(np.abs(B), ((0, pad), (0, 0)))
    absAc = (absA.reshape(A.shape[0], NG, L) @ Ca)                       # M x NG x lp1
    absBd = np.einsum("pt,gtn->gpn", Da, absB.reshape(NG, L, -1))        # NG x lp1 x N
    M, N = W.shape
    fA = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(L) + 2 * gamma(N) + 2 * gamma(lp1)
    fB = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(L) + 2 * gamma(M) + 2 * gamma(lp1)
    dAc_abs = np.einsum("mn,gpn->mgp", np.abs(W[rows]), absBd)           # |dY| |B_d|
    bA = fA * np.einsum("mgp,tp->mgt", dAc_abs, Ca).reshape(len(rows), NG * L)[:, :K]
    dBc_abs = np.einsum("mgp,mn->gpn", absAc, np.abs(W[:, cols]))        # |A_c|^T |dY|
    bB = fB * np.einsum("pt,gpn->gtn", Da, dBc_abs).reshape(NG * L, len(cols))[:K]
    return bA, bB


@pytest.mark.parametrize("M,N,K,Kb,R", [(300, 200, 512, 128, 32), (257, 129, 1000, 256, 64)])
def test_bf16_adjoint_matches_oracle(M, N, K, Kb, R):
    rng = np.random.default_rng(3)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    W = rng.normal(size=(M, N)).astype(np.float32)
    dA, dB = pj.proj_gemm_backward(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV),
                                   torch.from_numpy(W).to(DEV), Kb, R)
    A64, B64, W64 = (x.astype(np.float64) for x in (A, B, W))
    rA, rB = oracle.gemm_adjoint(A64, B64, W64, Kb, R)
    bA, bB = _bf16_grad_bounds(A64, B64, W64, Kb, R, 8, np.arange(M), np.arange(N))
    assert np.all(np.abs(dA.double().cpu().numpy() - rA) <= bA)
    assert np.all(np.abs(dB.double().cpu().numpy() - rB) <= bB)


@pytest.mark.parametrize("M,N,K,Kb,R", [(264, 136, 1000, 128, 32), (264, 136, 1001, 128, 64)])
def test_bf16_inputs_adjoint_matches_oracle(M, N, K, Kb, R):
    """BF16 A, B, dY and gradients: dY feeds both reduced products directly (the
    dB product reads A_c and dY MN-major), and K = 1001 leaves a last group of
    one value."""
    rng = np.random.default_rng(7)
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    W = torch.from_numpy(rng.normal(size=(M, N)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    dA, dB = pj.proj_gemm_backward(A, B, W, Kb, R)
    A64, B64, W64 = (x.double().cpu().numpy() for x in (A, B, W))
    rA, rB = oracle.gemm_adjoint(A64, B64, W64, Kb, R)
    bA, bB = _bf16_grad_bounds(A64, B64, W64, Kb, R, 8, np.arange(M), np.arange(N))
    gA, gB = dA.double().cpu().numpy(), dB.double().cpu().numpy()
    # gradients come back in BF16: allow one more rounding
    assert np.all(np.abs(gA - rA) <= bA + U_BF16 * (np.abs(rA) + bA))
    assert np.all(np.abs(gB - rB) <= bB + U_BF16 * (np.abs(rB) + bB))


def test_autograd_bf16_layer_sampled():
    """X 8192x4096 times W 4096x4096 in BF16 (std 0.02), block 256, R = 64: forward and backward."""
    X, Wt, dY = synth.layer_workload(seed=1)
    Xb = torch.from_numpy(X).to(DEV).to(torch.bfloat16).requires_grad_()
    Wb = torch.from_numpy(Wt).to(DEV).to(torch.bfloat16).requires_grad_()
    Y = pj.proj_matmul(Xb, Wb, 256, 64)
    g = torch.from_numpy(dY).to(DEV)
    Y.backward(g)
    rows = np.random.default_rng(4).choice(8192, 8, replace=False)
    cols = np.random.default_rng(5).choice(4096, 8, replace=False)
    X64 = Xb.detach().double().cpu().numpy()
    W64 = Wb.detach().double().cpu().numpy()
    # dY is rounded to BF16 by the backward (inputs are BF16)
    g64 = g.to(torch.bfloat16).double().cpu().numpy()
    # reference gradient rows / columns from the oracle's adjoint formula on the sampled slices:
    # dA[rows] depends on dY[rows] only; dB[:, cols] depends on dY[:, cols] only
    rA, _ = oracle.gemm_adjoint(X64[rows], W64, g64[rows], 256, 64)
    _, rB = oracle.gemm_adjoint(X64, W64[:, cols], g64[:, cols], 256, 64)
    bA, bB = _bf16_grad_bounds(X64, W64, g64, 256, 64, 8, rows, cols)
    gA = Xb.grad.double().cpu().numpy()[rows]
    gB = Wb.grad.double().cpu().numpy()[:, cols]
    # gradients come back in BF16: allow one more rounding
    assert np.all(np.abs(gA - rA) <= bA + U_BF16 * (np.abs(rA) + bA))
    assert np.all(np.abs(gB - rB) <= bB + U_BF16 * (np.abs(rB) + bB))


@pytest.mark.parametrize("M,N,K,Kb,R,out_dtype,pad", [
    (300, 200, 512, 128, 16, torch.float32, 0),       # l+1 = 1
    (257, 136, 1000, 128, 32, torch.bfloat16, 8),     # l+1 = 2, padded gradient rows
    (130, 264, 1001, 64, 32, torch.float32, 7),       # l+1 = 4, last group of one value
    (520, 384, 2048, 256, 256, torch.bfloat16, 0),    # l+1 = 8 (R = block)
    (64, 1024, 640, 128, 64, torch.float32, 4),       # l+1 = 4, one tile row of dY
    (512, 256, 2048, 256, 128, torch.float32, 0),     # both products in one 2-SM launch
    (384, 512, 1536, 256, 32, torch.bfloat16, 8),     # l+1 = 1, one 2-SM launch, padded rows
])
def test_bf16_adjoint_expanded_in_the_epilogue(M, N, K, Kb, R, out_dtype, pad):
    """L = 8 with l+1 in {1, 2, 4, 8} and 16-byte-aligned gradient rows: both reduced
    products map their components back to samples in the epilogue (dA through the
    lanes of a group, dB from each thread's own columns) and write the gradients
    themselves.  Ragged M, N, K and a short last group; gradients checked
    elementwise against the oracle's adjoint."""
    rng = np.random.default_rng(M + R)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    W = rng.normal(size=(M, N)).astype(np.float32)
    es = 2 if out_dtype == torch.bfloat16 else 4
    ka = -(-(K + pad) * es // 16) * 16 // es      # row pitches that keep 16-byte rows
    nb = -(-(N + pad) * es // 16) * 16 // es
    dA_buf = torch.full((M, ka), float("nan"), dtype=out_dtype, device=DEV)
    dB_buf = torch.full((K, nb), float("nan"), dtype=out_dtype, device=DEV)
    pj.proj_gemm_backward(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), torch.from_numpy(W).to(DEV),
                          Kb, R, out_dtype=out_dtype, dA=dA_buf[:, :K], dB=dB_buf[:, :N])
    torch.cuda.synchronize()
    # nothing is written past the gradients' columns
    if ka > K:
        assert torch.isnan(dA_buf[:, K:]).all()
    if nb > N:
        assert torch.isnan(dB_buf[:, N:]).all()
    A64, B64, W64 = (x.astype(np.float64) for x in (A, B, W))
    rA, rB = oracle.gemm_adjoint(A64, B64, W64, Kb, R)
    bA, bB = _bf16_grad_bounds(A64, B64, W64, Kb, R, 8, np.arange(M), np.arange(N))
    if out_dtype == torch.bfloat16:
        bA = bA + U_BF16 * (np.abs(rA) + bA)
        bB = bB + U_BF16 * (np.abs(rB) + bB)
    gA = dA_buf[:, :K].double().cpu().numpy()
    gB = dB_buf[:, :N].double().cpu().numpy()
    assert np.all(np.abs(gA - rA) <= bA), np.nanmax(np.abs(gA - rA) / bA)
    assert np.all(np.abs(gB - rB) <= bB), np.nanmax(np.abs(gB - rB) / bB)


@pytest.mark.parametrize("M,N,K,Kb,R,dtype,out_dtype", [
    (300, 200, 512, 128, 32, torch.float32, torch.float32),     # expansion in the epilogue, one 2-SM launch
    (257, 136, 1001, 128, 64, torch.bfloat16, torch.bfloat16),  # ragged, short last group
    (130, 264, 1000, 128, 48, torch.float32, torch.float32),    # l+1 = 3: the expansion kernels
    (96, 80, 300, 64, 16, torch.float64, torch.float64),        # FP64 throughout
])
def test_backward_from_saved_projections_is_identical(M, N, K, Kb, R, dtype, out_dtype):
    """proj_gemm_backward_saved reads A_c and B_d from the forward's workspace; the
    forward projected them with the same kernels the backward would use, so both
    gradients are bit-identical to proj_gemm_backward's."""
    rng = np.random.default_rng(M + N)
    A = torch.from_numpy(rng.normal(size=(M, K))).to(DEV).to(dtype)
    B = torch.from_numpy(rng.normal(size=(K, N))).to(DEV).to(dtype)
    W = torch.from_numpy(rng.normal(size=(M, N))).to(DEV).to(dtype)
    compute = "f64" if dtype == torch.float64 else "bf16"
    ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R, compute=compute), dtype=torch.uint8, device=DEV)
    pj.proj_gemm(A, B, Kb, R, compute=compute, workspace=ws)
    dA1, dB1 = pj.proj_gemm_backward(A, B, W, Kb, R, compute=compute, out_dtype=out_dtype)
    dA2, dB2 = pj.proj_gemm_backward_saved(ws, W, K, Kb, R, compute=compute, out_dtype=out_dtype)
    torch.cuda.synchronize()
    assert torch.equal(dA1, dA2) and torch.equal(dB1, dB2)
    # and against the oracle's adjoint (FP64: to rounding)
    if dtype == torch.float64:
        rA, rB = oracle.gemm_adjoint(A.cpu().numpy(), B.cpu().numpy(), W.cpu().numpy(), Kb, R)
        assert np.allclose(dA2.cpu().numpy(), rA, rtol=1e-11, atol=1e-11)
        assert np.allclose(dB2.cpu().numpy(), rB, rtol=1e-11, atol=1e-11)


def test_autograd_save_projections_matches_recompute():
    rng = np.random.default_rng(31)
    M, K, N = 512, 1024, 384
    X = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    Wt = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    g = torch.from_numpy(rng.normal(size=(M, N)).astype(np.float32)).to(DEV)
    grads = []
    for save in (False, True):
        Xr, Wr = X.clone().requires_grad_(), Wt.clone().requires_grad_()
        Y = pj.proj_matmul(Xr, Wr, 256, 64, save_projections=save)
        Y.backward(g)
        grads.append((Y.detach(), Xr.grad, Wr.grad))
    for a, b in zip(*grads):
        assert torch.equal(a, b)
    with pytest.raises(ValueError):
        pj.proj_matmul(X.clone().requires_grad_(), Wt, 256, 64, split=2, save_projections=True)


def test_backward_saved_rejects_a_small_forward_workspace():
    A = torch.zeros((64, 256), device=DEV)
    W = torch.zeros((64, 32), device=DEV)
    small = torch.empty(pj.gemm_workspace_size(64, 32, 256, 128, 32) - 256, dtype=torch.uint8, device=DEV)
    with pytest.raises(pj.ProjError):
        pj.proj_gemm_backward_saved(small, W, 256, 128, 32)
    del A
