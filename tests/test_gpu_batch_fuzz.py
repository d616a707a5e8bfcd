"""Seeded random batch plans: mixes of uneven GEMM instances (any l+1, plain or
split, BF16 or E4M3) and single-template correlations under random tunings
(CTA pairs or solo CTAs, round-robin or LPT order, fixed tile heights, splits
allowed or not), each instance checked against the FP64 oracle within its bound."""
import numpy as np
import pytest
import torch

import paper_1411_2860_gb300 as pj
from test_gpu_batch import _check_conv, _check_gemm, _conv_case, _desc, _gemm_case

pytestmark = pytest.mark.gpu

TUNINGS = [None, {"solo": 1}, {"schedule": 2}, {"max_split": 1}, {"tile_rows": 64}, {"schedule": 1, "solo": 1},
           {"us_per_tile": 50.0}]


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("seed", range(6))
def test_fuzz_batch(seed):
    rng = np.random.default_rng(3000 + seed)
    gemms = []
    for _ in range(int(rng.integers(4, 10))):
        Kb = int(rng.choice([64, 128, 256]))
        lp1 = int(rng.integers(1, 9))
        compute = "e4m3" if rng.random() < 0.25 else "bf16"
        split = int(rng.choice([1, 2]))
        gemms.append(_gemm_case(rng, int(rng.integers(1, 700)), int(rng.integers(1, 700)),
                                int(rng.integers(1, 3000)), Kb, lp1 * (Kb // 8), split, compute=compute))
    convs = [_conv_case(rng, int(rng.integers(1100, 30000)), 1024, 1, int(rng.choice([256, 512, 1024])),
                        seed=100 * seed + i) for i in range(int(rng.integers(0, 3)))]
    descs = [_desc(c) for c in gemms] + [pj.batch_conv(c["s"], c["k"], c["out"], c["R"]) for c in convs]
    order = rng.permutation(len(descs))
    tuning = TUNINGS[seed % len(TUNINGS)]
    plan = pj.BatchPlan([descs[i] for i in order], tuning=tuning)
    plan.run()
    plan.check()
    for c in gemms:
        _check_gemm(c)
    for i, c in enumerate(convs):
        _check_conv(c, seed=i)
