"""Batched launch (proj_batch_*): uneven GEMM and CONV instances in one grouped
persistent GEMM, each checked against the FP64 oracle within its bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
import synth
from helpers import (U_BF16, box_sums, conv_abs_entries, e4m3_scale_term, factor, factor_e4m3, gamma,
                     gemm_abs_parts, gemm_abs_product)

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _gemm_case(rng, M, N, K, Kb, R, split, kind="dct2", L=8, compute="bf16"):
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    Y = torch.full((M, N), float("nan"), device=DEV)
    return dict(A=A, B=B, Y=Y, Kb=Kb, R=R, split=split, kind=kind, L=L, compute=compute)


def _desc(c):
    return pj.batch_gemm(c["A"], c["B"], c["Y"], c["Kb"], c["R"], c["kind"], c["L"], c["split"],
                         compute=c["compute"])


def _check_gemm(c):
    A64 = c["A"].double().cpu().numpy()
    B64 = c["B"].double().cpu().numpy()
    ref = oracle.gemm_proj(A64, B64, c["Kb"], c["R"], c["kind"], c["L"])
    C, D = oracle.basis(c["kind"], c["L"])
    lp1 = c["R"] // (c["Kb"] // c["L"])
    nseg = 3 if c["split"] == 2 else 1
    if c["compute"] == "e4m3":
        absAc, absBd = gemm_abs_parts(A64, B64, c["L"], C, D, lp1)
        bound = factor_e4m3(absAc.shape[1] * nseg, c["L"], c["split"]) * (absAc @ absBd) + \
            e4m3_scale_term(absAc, absBd, c["split"])
    else:
        absprod, Kp = gemm_abs_product(A64, B64, c["L"], C, D, lp1)
        bound = factor(Kp * nseg, c["L"], c["split"]) * absprod
    got = c["Y"].double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound), np.nanmax(np.abs(got - ref) / bound)


def _conv_case(rng, S, T, nt, R, seed):
    s, k, _ = synth.audio_workload(S, T, nt, seed=seed)
    out = torch.full((S - T + 1, nt), float("nan"), device=DEV)
    return dict(s=torch.from_numpy(s).to(DEV), k=torch.from_numpy(k).to(DEV), out=out, R=R)


def _check_conv(c, n=1500, seed=0, split=1):
    s = c["s"].double().cpu().numpy()
    k = c["k"].double().cpu().numpy()
    T = k.shape[1]
    R = c["R"]
    lags = s.shape[0] - T + 1
    rng = np.random.default_rng(seed)
    mm = np.concatenate([rng.integers(0, lags, n), np.arange(max(0, lags - 300), lags)])
    tt = rng.integers(0, k.shape[0], len(mm))
    ref = oracle.conv_proj_entries(s, k, mm, tt, R, "haar", 64)
    if split == 2:   # hi.hi + hi.lo + lo.hi over three passes of the reduced K
        f = 4 * U_BF16 ** 2 + 2 * gamma(T // R) * (1 + U_BF16) ** 2 + 2 * gamma(3 * (R + 128)) * (1 + U_BF16) ** 2
    else:
        f = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(T // R) + 2 * gamma(R + 128)
    bound = f * conv_abs_entries(s, k, R, mm, tt)
    got = c["out"].double().cpu().numpy()
    assert not np.isnan(got).any()
    assert np.all(np.abs(got[mm, tt] - ref) <= bound), np.max(np.abs(got[mm, tt] - ref) / bound)


def test_mixed_batch_matches_oracle():
    rng = np.random.default_rng(0)
    gemms = [_gemm_case(rng, 300, 200, 1000, 128, 32, 1), _gemm_case(rng, 64, 513, 256, 128, 128, 2),
             _gemm_case(rng, 777, 130, 1536, 256, 64, 1), _gemm_case(rng, 129, 64, 3000, 512, 512, 2),
             _gemm_case(rng, 1, 1, 64, 64, 8, 1), _gemm_case(rng, 200, 300, 777, 64, 24, 1, "haar", 8)]
    convs = [_conv_case(rng, 20000, 1024, 1, 1024, 1), _conv_case(rng, 9000, 1024, 1, 512, 2),
             _conv_case(rng, 12345, 256, 3, 64, 3), _conv_case(rng, 4096, 1024, 2, 256, 4)]
    descs = [pj.batch_gemm(c["A"], c["B"], c["Y"], c["Kb"], c["R"], c["kind"], c["L"], c["split"]) for c in gemms]
    descs += [pj.batch_conv(c["s"], c["k"], c["out"], c["R"]) for c in convs]
    plan = pj.BatchPlan(descs)
    for _ in range(2):   # a second run of the same plan must give the same result
        plan.run()
        plan.check()
    for c in gemms:
        _check_gemm(c)
    for i, c in enumerate(convs):
        _check_conv(c, seed=i)


def test_batch_full_R_conv_matches_exact_and_single_call():
    rng = np.random.default_rng(1)
    c = _conv_case(rng, 60000, 1024, 1, 1024, 5)
    plan = pj.BatchPlan([pj.batch_conv(c["s"], c["k"], c["out"], 1024)])
    plan.run()
    plan.check()
    _check_conv(c)
    single = pj.proj_conv(c["s"], c["k"], 1024)
    assert oracle.rel_fro(c["out"].double().cpu().numpy(), single.double().cpu().numpy()) <= 2e-3


def test_batch_split_conv_matches_oracle_and_exact():
    """Correlation instances with the hi/lo split: within the split bound of the
    oracle, and at full R equal to the exact correlation to ~1e-5."""
    rng = np.random.default_rng(2)
    convs = [_conv_case(rng, 20000, 1024, 1, 1024, 6), _conv_case(rng, 9000, 1024, 2, 256, 7),
             _conv_case(rng, 5000, 256, 3, 64, 8)]
    g = _gemm_case(rng, 256, 130, 700, 128, 64, 2)
    descs = [pj.batch_conv(c["s"], c["k"], c["out"], c["R"], split=2) for c in convs]
    descs.append(pj.batch_gemm(g["A"], g["B"], g["Y"], g["Kb"], g["R"], split=2))
    plan = pj.BatchPlan(descs)
    plan.run()
    plan.check()
    for i, c in enumerate(convs):
        _check_conv(c, seed=10 + i, split=2)
    _check_gemm(g)
    c = convs[0]
    s = c["s"].double().cpu().numpy()
    k = c["k"].double().cpu().numpy()
    exact = np.stack([np.correlate(s, k[t], mode="valid") for t in range(k.shape[0])], axis=1)
    assert oracle.rel_fro(c["out"].double().cpu().numpy(), exact) <= 2e-5


def test_batch_rejects_bad_entry():
    A = torch.zeros((8, 64), device=DEV)
    B = torch.zeros((64, 8), device=DEV)
    Y = torch.zeros((8, 8), device=DEV)
    with pytest.raises(pj.ProjError):
        pj.BatchPlan([pj.batch_gemm(A, B, Y, 64, 5)])


def test_batch_e4m3_instances_match_oracle():
    """E4M3 GEMM instances (one and two terms, ragged shapes) beside BF16 GEMMs and a
    correlation: the E4M3 ones run in the block-scaled grouped launch."""
    rng = np.random.default_rng(3)
    gemms = [_gemm_case(rng, 300, 200, 1000, 128, 32, 1, compute="e4m3"),
             _gemm_case(rng, 64, 513, 256, 128, 128, 2, compute="e4m3"),
             _gemm_case(rng, 777, 130, 1536, 256, 64, 2, compute="e4m3"),
             _gemm_case(rng, 1, 1, 64, 64, 8, 1, compute="e4m3"),
             _gemm_case(rng, 250, 260, 900, 128, 64, 2)]
    conv = _conv_case(rng, 9000, 1024, 1, 512, 9)
    descs = [_desc(c) for c in gemms] + [pj.batch_conv(conv["s"], conv["k"], conv["out"], conv["R"])]
    plan = pj.BatchPlan(descs)
    info = plan.info()
    assert info["mx_tiles"] > 0 and info["gemm_tiles"] > 0
    plan.run()
    plan.check()
    for c in gemms:
        _check_gemm(c)
    _check_conv(conv, seed=20)


def _view(rng, rows, cols, dtype, pad, offset):
    """rows x cols with a row pitch of cols + pad elements, starting `offset` elements
    into its storage."""
    base = torch.from_numpy(rng.normal(size=offset + rows * (cols + pad)).astype(np.float32)).to(DEV).to(dtype)
    return base[offset:].view(rows, cols + pad)[:, :cols]


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_batch_operands_tma_cannot_address(dtype):
    """Operands whose row pitch or base is off the 16-byte grid (odd K or N, padded
    views, offset bases, K shorter than a tile, a short last group) are read by bulk
    copies of each row: BF16 and E4M3 instances, every l+1 class, with and without
    the split, against the oracle."""
    rng = np.random.default_rng(11)
    # M, N, K, pad and offset of A, pad and offset of B, block, R, split, compute
    shapes = [(300, 201, 1001, 0, 0, 0, 0, 128, 128, 2, "bf16"),
              (77, 130, 37, 3, 1, 5, 3, 64, 64, 1, "bf16"),
              (129, 64, 700, 1, 2, 0, 1, 128, 64, 1, "e4m3"),
              (513, 257, 2050, 0, 1, 0, 0, 256, 256, 2, "e4m3"),
              (1, 1, 9, 0, 0, 0, 0, 64, 64, 1, "bf16"),
              (40, 600, 300, 2, 0, 6, 0, 64, 16, 1, "bf16"),
              (100, 90, 333, 1, 1, 1, 1, 64, 24, 2, "bf16"),
              (33, 35, 515, 0, 3, 2, 0, 128, 128, 1, "e4m3")]
    gemms = []
    for M, N, K, pa, oa, pb, ob, Kb, R, split, compute in shapes:
        A = _view(rng, M, K, dtype, pa, oa)
        B = _view(rng, K, N, dtype, pb, ob)
        Y = torch.full((M, N), float("nan"), device=DEV)
        gemms.append(dict(A=A, B=B, Y=Y, Kb=Kb, R=R, split=split, kind="dct2", L=8, compute=compute))
    plan = pj.BatchPlan([_desc(c) for c in gemms])
    for _ in range(2):
        plan.run()
        plan.check()
    for c in gemms:
        _check_gemm(c)


def test_batch_e4m3_correlation_with_split_is_rejected():
    rng = np.random.default_rng(4)
    c = _conv_case(rng, 5000, 256, 1, 64, 10)
    d = pj.batch_conv(c["s"], c["k"], c["out"], c["R"], split=2, compute="e4m3")
    with pytest.raises(pj.ProjError):
        pj.BatchPlan([d])


def _check_conv_e4m3(c, n=1500, seed=0):
    """E4M3 bound of a lowered correlation: per reduced term the components carry
    2^-4 relative (plus 2^-16 from the BF16 hi + lo they are quantised from) and an
    absolute 2^-10 of their block's scale (< 2 max / 448) below the normal range."""
    s = c["s"].double().cpu().numpy()
    k = c["k"].double().cpu().numpy()
    T = k.shape[1]
    R = c["R"]
    Lb = T // R
    lags = s.shape[0] - T + 1
    rng = np.random.default_rng(seed)
    mm = np.concatenate([rng.integers(0, lags, n), np.arange(max(0, lags - 300), lags)])
    tt = rng.integers(0, k.shape[0], len(mm))
    ref = oracle.conv_proj_entries(s, k, mm, tt, R, "haar", 64)
    ue = 2.0 ** -4
    f = 2 * ue + ue ** 2 + 2 * 2.0 ** -16 + 2 * gamma(Lb) * (1 + ue) ** 2 + 2 * gamma(R + 256) * (1 + ue) ** 2
    bs = box_sums(np.abs(s), Lb) / np.sqrt(Lb)                     # |b| bounds
    kb = np.abs(k).reshape(k.shape[0], R, Lb).sum(axis=2) / np.sqrt(Lb)
    Mb, Mk = bs.max(), kb.max()
    v = 2.0 ** -10 / 224
    bsum = np.array([bs[m + Lb * np.arange(R)].sum() for m in mm])
    ksum = kb.sum(axis=1)[tt]
    bound = f * conv_abs_entries(s, k, R, mm, tt) + v * (1 + ue) * (Mb * ksum + Mk * bsum) + v * v * (R + 256) * Mb * Mk
    got = c["out"].double().cpu().numpy()
    assert not np.isnan(got).any()
    assert np.all(np.abs(got[mm, tt] - ref) <= bound), np.max(np.abs(got[mm, tt] - ref) / bound)
    return got[mm, tt], ref


@pytest.mark.parametrize("S,T,nt,R", [(20000, 1024, 1, 1024), (9000, 1024, 2, 512), (12000, 256, 3, 64)])
def test_batch_e4m3_correlation_matches_oracle(S, T, nt, R):
    """E4M3 correlations (the lowering on the block-scaled MMA: the signal phase
    quantised per block of 32, one scale per block shared by every window that
    reads it) beside a BF16 one, every lag phase and template checked against the
    oracle within the E4M3 bound."""
    rng = np.random.default_rng(S + R)
    c = _conv_case(rng, S, T, nt, R, 30 + nt)
    c2 = _conv_case(rng, 9000, 1024, 1, 512, 40)
    plan = pj.BatchPlan([pj.batch_conv(c["s"], c["k"], c["out"], R, compute="e4m3"),
                         pj.batch_conv(c2["s"], c2["k"], c2["out"], c2["R"])])
    assert plan.info()["mx_tiles"] > 0
    plan.run()
    plan.check()
    got, ref = _check_conv_e4m3(c, seed=S)
    _check_conv(c2, seed=41)
    # E4M3 carries ~2^-4 relative per component: the error is far above BF16's but bounded
    assert oracle.rel_fro(got, ref) <= 0.1


@pytest.mark.parametrize("compute,split,schedule", [("bf16", 1, 0), ("bf16", 2, 2), ("e4m3", 2, 0)])
def test_batch_tuner_splits_long_reduced_dimension(compute, split, schedule):
    """Few tiles with a long reduced dimension: the cost model cuts them into K
    pieces (partial products added into the zeroed FP32 output) and the result
    still meets the bound; the unsplit round-robin plan agrees with it."""
    rng = np.random.default_rng(5)
    cases = [_gemm_case(rng, 256, 256, 16384, 128, 128, split, compute=compute),
             _gemm_case(rng, 200, 130, 12000, 128, 64, split, compute=compute)]
    plan = pj.BatchPlan([_desc(c) for c in cases], tuning={"schedule": schedule})
    info = plan.info()
    assert info["split_instances"] == 2, info
    for _ in range(2):   # the zeroing runs every time: a second run must not accumulate
        plan.run()
        plan.check()
    for c in cases:
        _check_gemm(c)
    first = [c["Y"].clone() for c in cases]
    plain = pj.BatchPlan([_desc(c) for c in cases], tuning={"schedule": 1})
    assert plain.info()["split_instances"] == 0
    plain.run()
    plain.check()
    for c, y in zip(cases, first):
        _check_gemm(c)
        # only the FP32 summation order differs (K' up to 16384 terms)
        assert oracle.rel_fro(y.double().cpu().numpy(), c["Y"].double().cpu().numpy()) <= 1e-4


@pytest.mark.parametrize("tuning", [None, {"tile_rows": 64}, {"tile_rows": 96, "max_split": 1},
                                    {"schedule": 1}, {"schedule": 2}, {"us_per_tile": 50.0, "us_per_stage": 0.1},
                                    {"solo": 1}, {"solo": 1, "schedule": 2}])
def test_batch_tuning_knobs_give_the_same_products(tuning):
    rng = np.random.default_rng(6)
    gemms = [_gemm_case(rng, 300, 200, 1000, 128, 32, 1), _gemm_case(rng, 100, 513, 2560, 128, 128, 2),
             _gemm_case(rng, 33, 130, 1536, 256, 64, 1, compute="e4m3"),
             _gemm_case(rng, 520, 70, 4096, 128, 128, 2, compute="e4m3")]
    conv = _conv_case(rng, 9000, 1024, 1, 256, 11)
    descs = [_desc(c) for c in gemms] + [pj.batch_conv(conv["s"], conv["k"], conv["out"], conv["R"])]
    plan = pj.BatchPlan(descs, tuning=tuning)
    plan.run()
    plan.check()
    for c in gemms:
        _check_gemm(c)
    _check_conv(conv, seed=21)


def test_autotune_batch_measures_and_caches(tmp_path):
    rng = np.random.default_rng(7)
    gemms = [_gemm_case(rng, 300, 200, 2000, 128, 64, 1), _gemm_case(rng, 128, 256, 8192, 128, 128, 1)]
    descs = [_desc(c) for c in gemms]
    cache = str(tmp_path / "tune.json")
    best, trials = pj.autotune_batch(descs, reps=2, cache=cache)
    assert len(trials) == len(pj.DEFAULT_CANDIDATES)
    assert all(t["ms"] > 0 for t in trials)
    assert best == min(trials, key=lambda t: t["ms"])["tuning"]
    best2, trials2 = pj.autotune_batch(descs, reps=2, cache=cache)   # served from the cache
    assert best2 == best and trials2 == trials
    plan = pj.BatchPlan(descs, tuning=best)
    plan.run()
    plan.check()
    for c in gemms:
        _check_gemm(c)
