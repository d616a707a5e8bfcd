"""Failure detection on the GPU without a fault: bounded waits that run out.

The self-test kernels wait for something that never happens; each wait gives
up after its time limit and records its code in the workspace's error word,
the kernels drain what they issued and exit, pj_check reports PJ_ETIMEOUT, and
the same context then computes a correct product.
"""
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


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_gives_up_and_context_survives(which):
    assert pj.selftest_timeout(which) == pj.PJ_ETIMEOUT
    assert "bounded wait" in pj.last_error()
    # the context is still usable: a small product after the failed kernel is correct
    rng = np.random.default_rng(which)
    A, B = rng.normal(size=(130, 300)), rng.normal(size=(300, 260))
    Y = pj.proj_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 64, 32).cpu().numpy()
    assert oracle.rel_fro(Y, oracle.gemm_proj(A, B, 64, 32)) <= 1e-12


def test_selftest_rejects_unknown_kind():
    with pytest.raises(pj.ProjError):
        pj.selftest_timeout(2)
