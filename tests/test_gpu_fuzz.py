"""Seeded random shapes through the whole GPU path, against the FP64 oracle.

Each case draws its sizes, group size, kept projections, precision tier, input
dtype and row padding from its own seed, so tile counts (odd and even tile
columns, ragged last tiles, single-tile products) and the launch forms that
depend on them (CTA pairs, stream-K, per-group or TMA projection) vary from
case to case.  The bounds are the elementwise forward bounds of the fixed-shape
tests.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
import synth
from helpers import U_BF16, conv_abs_entries, factor, gamma, gemm_abs_parts

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _gemm_params(seed):
    rng = np.random.default_rng(1000 + seed)
    L = int(rng.choice([8, 8, 8, 4, 16]))
    groups = int(rng.choice([1, 2, 4, 8, 16, 32, 64]))
    Kb = L * groups
    lp1 = int(rng.integers(1, L + 1))
    R = lp1 * groups
    M, N = int(rng.integers(1, 700)), int(rng.integers(1, 700))
    K = int(rng.integers(1, 2500))
    split = int(rng.choice([1, 2]))
    lead = int(rng.integers(1, lp1)) if split == 2 and lp1 > 1 and rng.random() < 0.4 else 0
    in_dtype = torch.bfloat16 if rng.random() < 0.2 else torch.float32
    pad_a = int(rng.integers(1, 9)) if rng.random() < 0.3 else 0
    pad_b = int(rng.integers(1, 9)) if rng.random() < 0.3 else 0
    return dict(M=M, N=N, K=K, L=L, Kb=Kb, R=R, lp1=lp1, split=split, lead=lead, in_dtype=in_dtype,
                pad_a=pad_a, pad_b=pad_b)


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_bf16_gemm(seed):
    c = _gemm_params(seed)
    rng = np.random.default_rng(seed)
    M, N, K, L = c["M"], c["N"], c["K"], c["L"]
    Abig = torch.from_numpy(rng.normal(size=(M, K + c["pad_a"])).astype(np.float32)).to(DEV).to(c["in_dtype"])
    Bbig = torch.from_numpy(rng.normal(size=(K, N + c["pad_b"])).astype(np.float32)).to(DEV).to(c["in_dtype"])
    A, B = Abig[:, :K], Bbig[:, :N]
    Y = pj.proj_gemm(A, B, c["Kb"], c["R"], "dct2", L, split=c["split"], split_lead=c["lead"])
    Y = Y.double().cpu().numpy()
    A64, B64 = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, c["Kb"], c["R"], "dct2", L)
    C, D = oracle.basis("dct2", L)
    absAc, absBd = gemm_abs_parts(A64, B64, L, C, D, c["lp1"])
    Kp = absAc.shape[1]
    if c["lead"]:
        is_lead = (np.arange(Kp) % c["lp1"]) < c["lead"]
        g = 2 * gamma(L) * (1 + U_BF16) ** 2 + 2 * gamma(Kp + 2 * is_lead.sum()) * (1 + U_BF16) ** 2
        bound = ((4 * U_BF16 ** 2 + g) * (absAc[:, is_lead] @ absBd[is_lead])
                 + (2 * U_BF16 + U_BF16 ** 2 + g) * (absAc[:, ~is_lead] @ absBd[~is_lead]))
    else:
        bound = factor(Kp * (3 if c["split"] == 2 else 1), L, c["split"]) * (absAc @ absBd)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), f"{c}: worst ratio {np.max(err / bound):.3f}"


@pytest.mark.parametrize("seed", range(12))
def test_fuzz_conv(seed):
    rng = np.random.default_rng(2000 + seed)
    T = int(rng.choice([64, 128, 256, 512, 1024]))
    Lb = 2 ** int(rng.integers(0, int(np.log2(T // 64)) + 1))   # R = T / Lb, a multiple of 64
    R = T // Lb
    S = T + int(rng.integers(0, 6000))
    nt = int(rng.integers(1, 65))
    s, k, _ = synth.audio_workload(S, T, nt, seed=seed)
    got = pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), R).double().cpu().numpy()
    assert got.shape == (S - T + 1, nt)
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    n = min(1500, (S - T + 1) * nt)
    pick = np.random.default_rng(seed).choice((S - T + 1) * nt, size=n, replace=False)
    mm, tt = pick // nt, pick % nt
    ref = oracle.conv_proj_entries(s64, k64, mm, tt, R, "haar", 64)
    f = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(Lb) * (1 + U_BF16) ** 2 + 2 * gamma(R) * (1 + U_BF16) ** 2
    bound = f * conv_abs_entries(s64, k64, R, mm, tt)
    err = np.abs(got[mm, tt] - ref)
    assert np.all(err <= bound), f"S={S} T={T} nt={nt} R={R}: worst ratio {np.max(err / bound):.3f}"
