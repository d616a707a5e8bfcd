"""Projected GEMM on the GPU against the FP64 oracle (parity) and the exact product."""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
import synth
from helpers import U_BF16, factor, gamma, gemm_abs_parts, gemm_abs_product

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _user_C(L, seed=5):
    return np.random.default_rng(seed).normal(size=(L, L)) + 3 * np.eye(L)


# ------------------------------------------------------------------ basis --

@pytest.mark.parametrize("kind,L,lp1", [("dct2", 8, 1), ("dct2", 8, 3), ("dct2", 8, 8), ("dct2", 12, 5),
                                         ("haar", 64, 1), ("haar", 64, 16), ("haar", 64, 64), ("haar", 2, 1),
                                         ("user", 8, 3)])
def test_gpu_basis_matches_oracle(kind, L, lp1):
    uc = _user_C(L) if kind == "user" else None
    Cg, Dg = pj.basis_build(kind, L, lp1, uc)
    C, D = oracle.basis(kind, L, uc)
    tol = 1e-11 if kind == "user" else 1e-14
    np.testing.assert_allclose(Cg.cpu().numpy(), C[:, :lp1], atol=tol)
    np.testing.assert_allclose(Dg.cpu().numpy(), D[:lp1, :], atol=tol)


def test_gpu_basis_rejects_singular_user_matrix():
    with pytest.raises(pj.ProjError):
        pj.basis_build("user", 4, 2, np.ones((4, 4)))


# ------------------------------------------------------------ FP64 path --

@pytest.mark.parametrize("R", [128, 64, 32, 16])
def test_f64_uniform_256x512x256(R):
    """FP64 correctness workload: 256x512 by 512x256, block 128, DCT-II L=8."""
    A, B = synth.uniform_pair(256, 512, 256, seed=0)
    Y = pj.proj_gemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), 128, R).cpu().numpy()
    ref = oracle.gemm_proj(A, B, 128, R)
    assert oracle.rel_fro(Y, ref) <= 1e-12
    assert np.max(np.abs(Y - ref)) <= 1e-12 * np.max(np.abs(ref))
    if R == 128:
        assert oracle.rel_fro(Y, A @ B) <= 1e-12


@pytest.mark.parametrize("kind,L,Kb,R,K", [("dct2", 8, 64, 24, 300), ("haar", 8, 64, 16, 301),
                                            ("user", 8, 32, 12, 97), ("dct2", 16, 64, 64, 64),
                                            ("dct2", 4, 8, 2, 7)])
def test_f64_ragged(kind, L, Kb, R, K):
    rng = np.random.default_rng(1)
    M, N = 37, 53
    A, B = rng.normal(size=(M, K)), rng.normal(size=(K, N))
    uc = _user_C(L) if kind == "user" else None
    Y = pj.proj_gemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), Kb, R, kind, L,
                     user_C=uc).cpu().numpy()
    ref = oracle.gemm_proj(A, B, Kb, R, kind, L, uc)
    assert oracle.rel_fro(Y, ref) <= 1e-12


# ------------------------------------------------------------ BF16 path --

def _bf16_case(M, N, K, Kb, R, split, kind="dct2", L=8, in_dtype=torch.float32, out_dtype=torch.float32, seed=2):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    At = torch.from_numpy(A).to(DEV).to(in_dtype)
    Bt = torch.from_numpy(B).to(DEV).to(in_dtype)
    A64 = At.double().cpu().numpy()
    B64 = Bt.double().cpu().numpy()
    uc = _user_C(L) if kind == "user" else None
    Y = pj.proj_gemm(At, Bt, Kb, R, kind, L, split=split, out_dtype=out_dtype, user_C=uc)
    Y = Y.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, Kb, R, kind, L, uc)
    C, D = oracle.basis(kind, L, uc)
    lp1 = R // (Kb // L)
    absprod, Kp = gemm_abs_product(A64, B64, L, C, D, lp1)
    bound = factor(Kp * (3 if split == 2 else 1), L, split) * absprod
    if out_dtype == torch.bfloat16:
        bound += 2.0 ** -8 * (np.abs(ref) + bound)
    return Y, ref, bound


@pytest.mark.parametrize("M,N,K,Kb,R", [(300, 200, 1000, 128, 32), (256, 128, 512, 128, 128),
                                         (513, 257, 777, 64, 16), (1, 1, 8, 8, 8), (129, 300, 4096, 512, 64),
                                         (640, 384, 2048, 256, 256), (300, 516, 1000, 128, 64),
                                         (200, 301, 1000, 128, 128), (1000, 512, 640, 128, 64),
                                         (700, 256, 1000, 128, 128)])
@pytest.mark.parametrize("split", [1, 2])
def test_bf16_parity_elementwise(M, N, K, Kb, R, split):
    Y, ref, bound = _bf16_case(M, N, K, Kb, R, split)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"
    rel = oracle.rel_fro(Y, ref)
    assert rel <= (8e-3 if split == 1 else 2e-5), rel


@pytest.mark.parametrize("R", [24, 40, 56])
@pytest.mark.parametrize("in_dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("pad_a,pad_b", [(8, 12), (0, 0), (1, 3)])
def test_bf16_strided_operands_odd_components(R, in_dtype, pad_a, pad_b):
    """Row-padded views of wider buffers (lda > K, ldb > N), l+1 in {3, 5, 7},
    ragged M, N and K; pads that break 16-byte row alignment exercise the
    non-TMA projection path."""
    rng = np.random.default_rng(R + pad_a)
    M, N, K, Kb, split = 97, 520, 1100, 64, 2
    Abig = torch.from_numpy(rng.normal(size=(M, K + pad_a)).astype(np.float32)).to(DEV).to(in_dtype)
    Bbig = torch.from_numpy(rng.normal(size=(K, N + pad_b)).astype(np.float32)).to(DEV).to(in_dtype)
    A, B = Abig[:, :K], Bbig[:, :N]
    Y = pj.proj_gemm(A, B, Kb, R, split=split).double().cpu().numpy()
    A64, B64 = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, Kb, R, "dct2", 8)
    C, D = oracle.basis("dct2", 8)
    absprod, Kp = gemm_abs_product(A64, B64, 8, C, D, R // (Kb // 8))
    bound = factor(3 * Kp, 8, split) * absprod
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"


@pytest.mark.parametrize("kind,L,Kb,R", [("haar", 8, 64, 16), ("user", 8, 64, 24), ("dct2", 16, 128, 48)])
def test_bf16_other_bases(kind, L, Kb, R):
    Y, ref, bound = _bf16_case(200, 150, 333, Kb, R, 1, kind, L)
    assert np.all(np.abs(Y - ref) <= bound)


def test_bf16_inputs_and_outputs():
    Y, ref, bound = _bf16_case(300, 260, 640, 128, 64, 1, in_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    assert np.all(np.abs(Y - ref) <= bound)


def test_bf16_stream_k_schedule():
    """6 tiles of 939 K stages (split): the launch shares the stages of all tiles
    evenly over the SMs, cutting tiles between CTAs whose partial products are
    added into the zeroed output; the result still meets the elementwise bound."""
    Y, ref, bound = _bf16_case(300, 260, 20000, 128, 128, 2, seed=9)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"
    assert oracle.rel_fro(Y, ref) <= 2e-5


@pytest.mark.parametrize("M,N,K,Kb,R,lead", [(300, 200, 1000, 128, 128, 1), (513, 257, 777, 64, 32, 2),
                                              (256, 300, 2048, 512, 512, 4), (129, 64, 4100, 256, 192, 5),
                                              (250, 260, 700, 128, 64, 3)])
def test_bf16_split_lead_parity(M, N, K, Kb, R, lead):
    """Tiered split: only projections p < lead carry the lo term.  Each reduced
    component gets the bound of its own precision (4u^2 for the split ones,
    2u + u^2 for the plain ones)."""
    rng = np.random.default_rng(M + lead)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Y = pj.proj_gemm(At, Bt, Kb, R, split=2, split_lead=lead).double().cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = oracle.gemm_proj(A64, B64, Kb, R)
    C, D = oracle.basis("dct2", 8)
    lp1 = R // (Kb // 8)
    absAc, absBd = gemm_abs_parts(A64, B64, 8, C, D, lp1)
    is_lead = (np.arange(absAc.shape[1]) % lp1) < lead
    lead_part = absAc[:, is_lead] @ absBd[is_lead]
    tail_part = absAc[:, ~is_lead] @ absBd[~is_lead]
    Kp = absAc.shape[1]
    g = 2 * gamma(8) * (1 + U_BF16) ** 2 + 2 * gamma(Kp + 2 * is_lead.sum()) * (1 + U_BF16) ** 2
    bound = (4 * U_BF16 ** 2 + g) * lead_part + (2 * U_BF16 + U_BF16 ** 2 + g) * tail_part
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3f}"
    # with every projection split it is the plain split product
    if lead >= lp1:
        return
    Yall = pj.proj_gemm(At, Bt, Kb, R, split=2, split_lead=lp1).double().cpu().numpy()
    Y0 = pj.proj_gemm(At, Bt, Kb, R, split=2).double().cpu().numpy()
    assert np.array_equal(Yall, Y0)


def test_split_lead_rejected_without_split():
    A = torch.zeros((8, 64), device=DEV)
    with pytest.raises(pj.ProjError):
        pj.proj_gemm(A, torch.zeros((64, 8), device=DEV), 64, 64, split=1, split_lead=1)


def test_full_R_matches_exact_product_to_bf16_accuracy():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(512, 1024)).astype(np.float32)
    B = rng.normal(size=(1024, 256)).astype(np.float32)
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    ex = A.astype(np.float64) @ B.astype(np.float64)
    y1 = pj.proj_gemm(At, Bt, 128, 128, split=1).double().cpu().numpy()
    y2 = pj.proj_gemm(At, Bt, 128, 128, split=2).double().cpu().numpy()
    assert oracle.rel_fro(y1, ex) <= 6e-3
    assert oracle.rel_fro(y2, ex) <= 1e-5


# ------------------------------------------------------------ edge cases --

def test_zero_inner_dimension_gives_zeros():
    A = torch.zeros((5, 0), device=DEV)
    B = torch.zeros((0, 7), device=DEV)
    Y = pj.proj_gemm(A, B, 64, 8)
    assert Y.shape == (5, 7) and torch.all(Y == 0)


def test_empty_outputs_are_noops():
    Y = pj.proj_gemm(torch.zeros((0, 64), device=DEV), torch.zeros((64, 9), device=DEV), 64, 8)
    assert Y.shape == (0, 9)


def test_invalid_R_raises_on_gpu():
    A = torch.zeros((4, 64), device=DEV)
    with pytest.raises(pj.ProjError):
        pj.proj_gemm(A, torch.zeros((64, 4), device=DEV), 64, 5)


def test_staged_project_then_multiply_matches_single_call():
    rng = np.random.default_rng(4)
    A = torch.from_numpy(rng.normal(size=(300, 512)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(512, 200)).astype(np.float32)).to(DEV)
    Y1 = pj.proj_gemm(A, B, 128, 32)
    ws = torch.empty(pj.gemm_workspace_size(300, 200, 512, 128, 32), dtype=torch.uint8, device=DEV)
    pj.proj_gemm_project(A, B, 128, 32, ws)
    Y2 = torch.empty((300, 200), device=DEV)
    pj.proj_gemm_multiply(Y2, 512, 128, 32, ws)
    pj.check(ws)
    assert torch.equal(Y1, Y2)


def test_host_buffers_round_trip():
    rng = np.random.default_rng(6)
    A = torch.from_numpy(rng.normal(size=(64, 256)).astype(np.float32)).pin_memory()
    B = torch.from_numpy(rng.normal(size=(256, 96)).astype(np.float32)).pin_memory()
    Y = pj.proj_gemm(A, B, 64, 16)
    assert Y.device.type == "cpu"
    Yd = pj.proj_gemm(A.to(DEV), B.to(DEV), 64, 16).cpu()
    assert torch.equal(Y, Yd)


# --------------------------------------------- face-matching-shaped GEMM --

@pytest.fixture(scope="module")
def face_inputs():
    A = synth.face_probes(4096, seed=0)
    B = synth.orthonormal_features(10304, 2048, seed=1)
    return A, B


@pytest.mark.parametrize("R,split", [(512, 2), (512, 1), (128, 1), (64, 1)])
def test_face_gemm_sampled_parity(face_inputs, R, split):
    """4096 x 10304 by 10304 x 2048, block 512 (20 full blocks + a 64-wide tail)."""
    A, B = face_inputs
    Y = pj.proj_gemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), 512, R, split=split)
    rng = np.random.default_rng(7)
    ii = rng.integers(0, 4096, 256)
    jj = rng.integers(0, 2048, 256)
    got = Y[torch.from_numpy(ii).to(DEV), torch.from_numpy(jj).to(DEV)].double().cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = oracle.gemm_proj_entries(A64, B64, ii, jj, 512, R)
    C, D = oracle.basis("dct2", 8)
    absprod, Kp = gemm_abs_product(A64[ii], B64[:, jj], 8, C, D, R // 64)
    bound = factor(Kp * (3 if split == 2 else 1), 8, split) * np.diag(absprod)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


@pytest.mark.parametrize("compute,split,lead", [("bf16", 1, 0), ("bf16", 2, 1), ("e4m3", 2, 0)])
def test_pre_projected_operand_reuse(compute, split, lead):
    """A fixed B (a feature or weight matrix) is projected once; every new A is
    projected alone and multiplied with the cached B_d.  Each product equals the
    one-call proj_gemm of the same operands bit for bit."""
    rng = np.random.default_rng(21)
    M, K, N = 300, 1500, 260
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    ws = torch.empty(pj.gemm_workspace_size(M, N, K, 128, 64, compute=compute, split=split, split_lead=lead),
                     dtype=torch.uint8, device=DEV)
    pj.proj_gemm_project(None, B, 128, 64, ws, compute=compute, split=split, M=M, N=N, K=K, split_lead=lead)
    for seed in range(3):
        A = torch.from_numpy(np.random.default_rng(seed).normal(size=(M, K)).astype(np.float32)).to(DEV)
        pj.proj_gemm_project(A, None, 128, 64, ws, compute=compute, split=split, N=N, split_lead=lead)
        Y = torch.empty((M, N), device=DEV)
        pj.proj_gemm_multiply(Y, K, 128, 64, ws, compute=compute, split=split, split_lead=lead)
        pj.check(ws)
        ref = pj.proj_gemm(A, B, 128, 64, compute=compute, split=split, split_lead=lead)
        assert torch.equal(Y, ref)


def test_learned_pca_basis_parity():
    """A user basis learned from the data (principal axes of A's 8-sample groups)
    through PJ_BASIS_USER: GPU against the oracle with the same basis."""
    A = synth.face_probes(300, seed=5)
    B = np.random.default_rng(6).normal(size=(A.shape[1], 200)).astype(np.float32)
    G = A.astype(np.float64).reshape(-1, 8)
    w, V = np.linalg.eigh(G.T @ G / G.shape[0])
    C = V[:, ::-1].copy()
    Y = pj.proj_gemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), 512, 128, "user", 8,
                     user_C=C).double().cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = oracle.gemm_proj(A64, B64, 512, 128, "user", 8, C)
    Cb, Db = oracle.basis("user", 8, C)
    absprod, Kp = gemm_abs_product(A64, B64, 8, Cb, Db, 2)
    bound = factor(Kp, 8, 1) * absprod
    assert np.all(np.abs(Y - ref) <= bound)


def test_user_basis_in_a_captured_graph():
    """The user matrix is read when the stream runs the call: a captured graph
    replays the staged calls with the matrix the binding keeps on the workspace."""
    rng = np.random.default_rng(22)
    A = torch.from_numpy(rng.normal(size=(256, 1024)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(1024, 200)).astype(np.float32)).to(DEV)
    C = _user_C(8)
    ref = pj.proj_gemm(A, B, 128, 32, "user", 8, user_C=C)
    ws = torch.empty(pj.gemm_workspace_size(256, 200, 1024, 128, 32, "user", 8, user_C=C), dtype=torch.uint8,
                     device=DEV)
    Y = torch.empty((256, 200), device=DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pj.proj_gemm_project(A, B, 128, 32, ws, "user", 8, user_C=C, stream=s)
        pj.proj_gemm_multiply(Y, 1024, 128, 32, ws, "user", 8, user_C=C, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            pj.proj_gemm_project(A, B, 128, 32, ws, "user", 8, user_C=C, stream=s)
            pj.proj_gemm_multiply(Y, 1024, 128, 32, ws, "user", 8, user_C=C, stream=s)
    import gc
    gc.collect()
    Y.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(Y, ref)
