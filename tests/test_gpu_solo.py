"""The "solo" library build (no CTA pairs, no multicast form), which a process
running one of several GPUs loads, computes what the one-GPU build computes.

One process loads one build, so the solo library runs in a child process: it
forms a BF16 projected GEMM whose tile columns pair up (the one-GPU build runs
it on CTA pairs) and an E4M3 one, and writes them to a file; this process
compares them elementwise with the FP64 oracle under the same bounds as the
other parity tests, and checks that the child loaded the solo build.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from helpers import factor, gemm_abs_product

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1411_2860_gb300 as pj
pj.select_library("solo")
pj.build()
A = torch.from_numpy(np.load(sys.argv[2] + "/A.npy")).cuda()
B = torch.from_numpy(np.load(sys.argv[2] + "/B.npy")).cuda()
Y = pj.proj_gemm(A, B, 256, 64, split=2)
Y8 = pj.proj_gemm(A, B, 256, 64, compute="e4m3", split=2)
torch.cuda.synchronize()
np.save(sys.argv[2] + "/Y.npy", Y.double().cpu().numpy())
np.save(sys.argv[2] + "/Y8.npy", Y8.double().cpu().numpy())
open(sys.argv[2] + "/version.txt", "w").write(pj._load().pj_version().decode())
"""


def test_solo_build_matches_oracle(tmp_path):
    rng = np.random.default_rng(21)
    M, N, K = 520, 1024, 1300          # 8 tile columns: CTA pairs in the one-GPU build
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    np.save(tmp_path / "A.npy", A)
    np.save(tmp_path / "B.npy", B)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "solo" in (tmp_path / "version.txt").read_text()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = oracle.gemm_proj(A64, B64, 256, 64, "dct2", 8)
    C, D = oracle.basis("dct2", 8)
    absprod, Kp = gemm_abs_product(A64, B64, 8, C, D, 2)
    Y = np.load(tmp_path / "Y.npy")
    assert np.all(np.abs(Y - ref) <= factor(3 * Kp, 8, 2) * absprod)
    Y8 = np.load(tmp_path / "Y8.npy")
    assert oracle.rel_fro(Y8, ref) <= 5e-3
