"""proj_conv_noalloc, the entry point for callers that cannot allocate device memory.

It must give what proj_conv gives with a caller workspace, call after call,
from its static scratch area, and refuse problems larger than that area.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
import synth
from helpers import U_BF16, conv_abs_entries, gamma

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def noalloc():
    pj.build()
    lib = pj._load()
    fn = lib.proj_conv_noalloc
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    fn.argtypes = [vp, i64, vp, i64, i64, vp, i32, i32, i64, i64, ctypes.POINTER(pj._Basis),
                   ctypes.POINTER(pj._Prec), vp]
    fn.restype = ctypes.c_int
    return fn


def _call(fn, sig, tpl, out, R):
    S, (nt, T) = sig.shape[0], tpl.shape
    b = pj._Basis(pj.BASIS["haar"], 64, None)
    p = pj._Prec(pj.PJ_BF16, 1, 0, 0)
    return fn(ctypes.c_void_p(sig.data_ptr()), S, ctypes.c_void_p(tpl.data_ptr()), T, nt,
              ctypes.c_void_p(out.data_ptr()), pj.PJ_F32, pj.PJ_F32, T, R, ctypes.byref(b), ctypes.byref(p),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(noalloc):
    cases = [(60000, 1024, 64, 256, 0), (1 << 20, 4096, 64, 4096, 1), (30000, 4096, 17, 1024, 2)]
    for S, T, nt, R, seed in cases:
        s, k, _ = synth.audio_workload(S, T, nt, seed=seed)
        sig, tpl = torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV)
        ref = pj.proj_conv(sig, tpl, R)
        out = torch.full_like(ref, float("nan"))
        assert _call(noalloc, sig, tpl, out, R) == 0, pj.last_error()
        torch.cuda.synchronize()
        rng = np.random.default_rng(seed)
        mm = rng.integers(0, S - T + 1, 2000)
        tt = rng.integers(0, nt, 2000)
        f = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(T // R) + 2 * gamma(R)
        bound = f * conv_abs_entries(s.astype(np.float64), k.astype(np.float64), R, mm, tt)
        a = out.cpu().numpy()
        b = ref.cpu().numpy()
        assert np.all(np.abs(a[mm, tt] - b[mm, tt]) <= bound)
        assert torch.equal(out, ref)


def test_noalloc_result_matches_oracle(noalloc):
    s, k, _ = synth.audio_workload(10000, 1024, 8, seed=3)
    sig, tpl = torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV)
    out = torch.empty((10000 - 1024 + 1, 8), device=DEV)
    for _ in range(2):
        assert _call(noalloc, sig, tpl, out, 512) == 0, pj.last_error()
    ref = oracle.conv_proj(s.astype(np.float64), k.astype(np.float64), 512, "haar", 64)
    assert oracle.rel_fro(out.double().cpu().numpy(), ref) <= 4e-3


def test_noalloc_refuses_problems_beyond_its_area(noalloc):
    S = 3 << 20                      # about 50 MB of scratch at full R
    sig = torch.zeros(S, device=DEV)
    tpl = torch.zeros((64, 4096), device=DEV)
    out = torch.empty((1, 64), device=DEV)   # never written: the call must stop before launching
    st = _call(noalloc, sig, tpl, out, 4096)
    assert st == pj.PJ_ENOMEM
    assert "20 MiB" in pj.last_error()
