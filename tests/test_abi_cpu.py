"""The C ABI without a GPU: the library loads, exports every function declared
in include/*.h, and rejects invalid arguments before touching CUDA."""
import ctypes

import pytest

import paper_1411_2860_gb300 as pj


@pytest.fixture(scope="module")
def lib():
    pj.build()
    return pj._load()


def test_exports_every_declared_symbol(lib):
    names = pj.exported_symbols()
    for expected in ("proj_gemm", "proj_conv", "proj_gemm_backward", "pj_last_error", "pj_check",
                     "proj_gemm_workspace_size", "proj_conv_workspace_size", "pj_basis_build"):
        assert expected in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/*.h but not exported"


def _b(kind=0, L=8):
    return pj._Basis(kind, L, None)


def _p(compute=pj.PJ_BF16, split=1):
    return pj._Prec(compute, split, 0, 0)


@pytest.mark.parametrize("block_k,R,kind,L,split,why", [
    (128, 20, 0, 8, 1, "R not a multiple of block_k/L"),
    (100, 16, 0, 8, 1, "block_k not a multiple of L"),
    (128, 256, 0, 8, 1, "R larger than the block"),
    (128, 16, 7, 8, 1, "unknown basis"),
    (128, 16, 1, 12, 1, "Haar with L not a power of two"),
    (128, 16, 0, 80, 1, "L above 64"),
    (128, 16, 0, 8, 3, "split_terms 3"),
    (128, 16, 2, 8, 1, "user basis without a matrix"),
])
def test_gemm_validation_rejects(lib, block_k, R, kind, L, split, why):
    b, p = _b(kind, L), _p(split=split)
    assert lib.proj_gemm_workspace_size(64, 64, 256, block_k, R, ctypes.byref(b), ctypes.byref(p)) == 0, why
    buf = ctypes.create_string_buffer(1024)
    st = lib.proj_gemm(buf, 256, buf, 64, buf, 64, 64, 64, 256, pj.PJ_F32, pj.PJ_F32, block_k, R, ctypes.byref(b),
                       ctypes.byref(p), None, 0, None)
    assert st == pj.PJ_EINVAL, (why, pj.last_error())
    assert pj.last_error()


def test_gemm_dtype_and_workspace_checks(lib):
    b, p = _b(), _p()
    n = lib.proj_gemm_workspace_size(300, 200, 1000, 128, 32, ctypes.byref(b), ctypes.byref(p))
    assert n > 0
    buf = ctypes.create_string_buffer(64)
    # F64 input with BF16 compute is unsupported
    st = lib.proj_gemm(buf, 1000, buf, 200, buf, 200, 300, 200, 1000, pj.PJ_F64, pj.PJ_F32, 128, 32,
                       ctypes.byref(b), ctypes.byref(p), None, 0, None)
    assert st == pj.PJ_EUNSUPPORTED
    # NULL workspace
    st = lib.proj_gemm(ctypes.c_void_p(256), 1000, ctypes.c_void_p(256), 200, ctypes.c_void_p(256), 200, 300, 200,
                       1000, pj.PJ_F32, pj.PJ_F32, 128, 32, ctypes.byref(b), ctypes.byref(p), None, 0, None)
    assert st == pj.PJ_EINVAL
    # too-small workspace
    st = lib.proj_gemm(ctypes.c_void_p(256), 1000, ctypes.c_void_p(256), 200, ctypes.c_void_p(256), 200, 300, 200,
                       1000, pj.PJ_F32, pj.PJ_F32, 128, 32, ctypes.byref(b), ctypes.byref(p), ctypes.c_void_p(4096),
                       16, None)
    assert st == pj.PJ_ENOMEM
    # lda < K
    st = lib.proj_gemm(ctypes.c_void_p(256), 999, ctypes.c_void_p(256), 200, ctypes.c_void_p(256), 200, 300, 200,
                       1000, pj.PJ_F32, pj.PJ_F32, 128, 32, ctypes.byref(b), ctypes.byref(p), ctypes.c_void_p(4096),
                       n, None)
    assert st == pj.PJ_EINVAL


def test_workspace_size_grows_with_split_and_R(lib):
    b = _b()
    n1 = lib.proj_gemm_workspace_size(4096, 2048, 10304, 512, 64, ctypes.byref(b), ctypes.byref(_p()))
    n2 = lib.proj_gemm_workspace_size(4096, 2048, 10304, 512, 64, ctypes.byref(b), ctypes.byref(_p(split=2)))
    n3 = lib.proj_gemm_workspace_size(4096, 2048, 10304, 512, 512, ctypes.byref(b), ctypes.byref(_p()))
    assert 0 < n1 < n2 and n1 < n3
    # reduced inner dimension: 20 full blocks of 8 components + 64-wide tail with 8*1 -> 168, padded to 192
    assert n1 >= 2 * 192 * (4096 + 2048)


@pytest.mark.parametrize("S,T,nt,block,R,kind,L,why,code", [
    (10000, 1024, 4, 512, 256, 1, 64, "block != T", pj.PJ_EINVAL),
    (1000, 1024, 4, 1024, 256, 1, 64, "T > S", pj.PJ_EINVAL),
    (10000, 1024, 4, 1024, 100, 1, 64, "R not (l+1)T/L", pj.PJ_EINVAL),
    (10000, 1024, 4, 1024, 384, 0, 8, "DCT with l+1 = 3, not a power of two", pj.PJ_EUNSUPPORTED),
    (10000, 1024, 65, 1024, 256, 1, 64, "more than 64 templates", pj.PJ_EUNSUPPORTED),
    (10000, 1024, 4, 1024, 768, 1, 64, "l+1 = 48 not a power of two", pj.PJ_EUNSUPPORTED),
    (10000, 1000, 4, 1000, 1000, 1, 7, "Haar with L = 7", pj.PJ_EINVAL),
])
def test_conv_validation(lib, S, T, nt, block, R, kind, L, why, code):
    b, p = _b(kind, L), _p()
    assert lib.proj_conv_workspace_size(S, T, nt, block, R, ctypes.byref(b), ctypes.byref(p)) == 0, why
    st = lib.proj_conv(ctypes.c_void_p(256), S, ctypes.c_void_p(256), T, nt, ctypes.c_void_p(256), pj.PJ_F32,
                       pj.PJ_F32, block, R, ctypes.byref(b), ctypes.byref(p), ctypes.c_void_p(4096), 1 << 40, None)
    assert st == code, (why, pj.last_error())


def test_conv_any_basis_geometry(lib):
    """The general path takes any basis with l+1 a power of two, and templates whose length
    is not a multiple of 64 (the last 64-component chunk is padded with zeros)."""
    p = _p()
    for kind, L, T, R in ((0, 8, 1024, 512), (0, 8, 200, 200), (0, 16, 1024, 1024), (1, 8, 1000, 1000),
                          (0, 64, 640, 640)):
        b = _b(kind, L)
        assert lib.proj_conv_workspace_size(10000, T, 4, T, R, ctypes.byref(b), ctypes.byref(p)) > 0, (kind, L, T, R)
    # DCT-II at L = 8 and l+1 = 8: one copy of eight phases of the projected signal
    n_dct = lib.proj_conv_workspace_size(1 << 20, 4096, 64, 4096, 4096, ctypes.byref(_b(0, 8)), ctypes.byref(p))
    assert 16 << 20 <= n_dct <= 20 << 20


def test_conv_workspace_size_config2(lib):
    b, p = _b(1, 64), _p()
    n = lib.proj_conv_workspace_size(1 << 20, 4096, 64, 4096, 4096, ctypes.byref(b), ctypes.byref(p))
    # eight shifted BF16 copies of the signal dominate: about 16 MiB
    assert 16 << 20 <= n <= 20 << 20


def test_backward_is_declared(lib):
    assert hasattr(lib, "proj_gemm_backward")


def _fake_batch_desc(M=300, N=200, K=1000, block=128, R=32, compute=pj.PJ_BF16):
    """A GEMM batch descriptor with placeholder device addresses (sizing reads no data)."""
    b, _ = pj._basis("dct2", 8)
    return pj._BatchDesc(0, pj.PJ_F32, pj.PJ_F32, 0, 1 << 20, 2 << 20, 3 << 20, M, N, K, K, N, N, block, R, b,
                         pj._Prec(compute, 1, 0, 0))


def test_batch_tuning_validation(lib):
    arr = (pj._BatchDesc * 2)(_fake_batch_desc(), _fake_batch_desc(2048, 2048, 8192, compute=pj.PJ_E4M3))
    base = lib.proj_batch_workspace_size(arr, 2)
    assert base > 0
    assert lib.proj_batch_workspace_size_tuned(arr, 2, None) == base
    for bad in ({"tile_rows": 48}, {"tile_rows": 512}, {"schedule": 3}, {"max_split": 100},
                {"us_per_stage": -1.0}, {"solo": 2}):
        t = pj._tuning(bad)
        assert lib.proj_batch_workspace_size_tuned(arr, 2, ctypes.byref(t)) == 0, bad
    # smaller tiles need more scale blocks and tile entries; no split needs the fewest
    small = pj._tuning({"tile_rows": 32})
    nosplit = pj._tuning({"max_split": 1})
    assert lib.proj_batch_workspace_size_tuned(arr, 2, ctypes.byref(small)) > base
    assert lib.proj_batch_workspace_size_tuned(arr, 2, ctypes.byref(nosplit)) < base
    with pytest.raises(ValueError):
        pj._tuning({"tiles": 3})


def test_report_and_selftest_validate_before_cuda(lib):
    rep = pj._Report()
    b, p = _b(), _p()
    fake = ctypes.c_void_p(256 * 1024)  # never dereferenced: validation fails first
    # no report to fill
    assert lib.proj_gemm_report(fake, 64, fake, 64, 64, 64, 64, pj.PJ_F32, pj.PJ_F32, 64, 16, ctypes.byref(b),
                                ctypes.byref(p), fake, 1 << 20, None, None) == pj.PJ_EINVAL
    # R not a multiple of block_k / L
    assert lib.proj_gemm_report(fake, 64, fake, 64, 64, 64, 64, pj.PJ_F32, pj.PJ_F32, 64, 12, ctypes.byref(b),
                                ctypes.byref(p), fake, 1 << 20, None, ctypes.byref(rep)) == pj.PJ_EINVAL
    # lda shorter than a row of A
    assert lib.proj_gemm_report(fake, 32, fake, 64, 64, 64, 64, pj.PJ_F32, pj.PJ_F32, 64, 16, ctypes.byref(b),
                                ctypes.byref(p), fake, 1 << 20, None, ctypes.byref(rep)) == pj.PJ_EINVAL
    # workspace too small
    assert lib.proj_gemm_report(fake, 64, fake, 64, 64, 64, 64, pj.PJ_F32, pj.PJ_F32, 64, 16, ctypes.byref(b),
                                ctypes.byref(p), fake, 16, None, ctypes.byref(rep)) == pj.PJ_ENOMEM
    assert lib.proj_gemm_report_workspace_size(-1, 64) == 0
    assert lib.proj_gemm_report_workspace_size(1000, 128) > lib.proj_gemm_report_workspace_size(100, 128) > 0
    # the self-test only knows kinds 0 and 1, and needs its workspace
    assert lib.pj_selftest_workspace_size() > 0
    assert lib.pj_selftest_timeout(2, fake, 1 << 24, None) == pj.PJ_EINVAL
    assert lib.pj_selftest_timeout(0, fake, 16, None) == pj.PJ_ENOMEM


def test_tuning_cache_is_versioned_and_checksummed(tmp_path, lib):
    import json
    cache = str(tmp_path / "tune.json")
    best, trials = {"schedule": 1}, [{"tuning": {"schedule": 1}, "ms": 1.5, "info": {}}]
    assert pj._cache_load(cache, "k") is None                      # no file
    pj._cache_store(cache, "k", best, trials)
    assert pj._cache_load(cache, "k") == (best, trials)
    assert pj._cache_load(cache, "other") is None
    data = json.load(open(cache))
    data["k"]["trials"][0]["ms"] = 0.1                              # edited entry: checksum fails
    json.dump(data, open(cache, "w"))
    assert pj._cache_load(cache, "k") is None
    pj._cache_store(cache, "k", best, trials)
    data = json.load(open(cache))
    data["k"]["version"] = pj.TUNE_CACHE_VERSION + 1                # another cache version
    json.dump(data, open(cache, "w"))
    assert pj._cache_load(cache, "k") is None
    open(cache, "w").write("{not json")                            # corrupt file: ignored, then replaced
    assert pj._cache_load(cache, "k") is None
    pj._cache_store(cache, "k", best, trials)
    assert pj._cache_load(cache, "k") == (best, trials)


def test_fp8_tier_validation(lib):
    """The FP8 tier of truncated projections (pj_precision.fp8_tier) is checked before
    anything touches CUDA: l+1 + tier within L, BF16 compute only, FP32 output, and
    not offered by the calls that have no tier (backward, CONV, batch, report)."""
    b = _b()

    def prec(tier, compute=pj.PJ_BF16, split=1, lead=0):
        return pj._Prec(compute, split, lead, tier)

    ok = lib.proj_gemm_workspace_size(300, 200, 1000, 128, 32, ctypes.byref(b), ctypes.byref(prec(6)))
    base = lib.proj_gemm_workspace_size(300, 200, 1000, 128, 32, ctypes.byref(b), ctypes.byref(prec(0)))
    assert ok > base > 0                                   # the tier's E4M3 operands live after the BF16 ones
    for bad, why in ((prec(7), "l+1 = 2 plus 7 > L = 8"), (prec(-1), "negative tier"),
                     (prec(2, compute=pj.PJ_E4M3), "tier on E4M3 compute"),
                     (prec(2, compute=pj.PJ_F64), "tier on FP64 compute")):
        assert lib.proj_gemm_workspace_size(300, 200, 1000, 128, 32, ctypes.byref(b), ctypes.byref(bad)) == 0, why
    buf = ctypes.create_string_buffer(64)
    fake_ws = ctypes.c_void_p(1 << 20)     # aligned and large enough on paper; validation fails before any use
    st = lib.proj_gemm(buf, 1000, buf, 200, buf, 200, 300, 200, 1000, pj.PJ_F32, pj.PJ_BF16, 128, 32,
                       ctypes.byref(b), ctypes.byref(prec(6)), fake_ws, ok, None)
    assert st == pj.PJ_EUNSUPPORTED and "FP32" in pj.last_error()
    assert lib.proj_gemm_backward_workspace_size(300, 200, 1000, 128, 32, ctypes.byref(b), ctypes.byref(prec(2))) == 0
    hb = _b(1, 64)
    assert lib.proj_conv_workspace_size(10000, 1024, 4, 1024, 256, ctypes.byref(hb), ctypes.byref(prec(2))) == 0


def test_backward_saved_validation(lib):
    """proj_gemm_backward_saved checks its forward workspace before anything touches
    CUDA: NULL, smaller than the forward of this product needs, or the same buffer
    as its own workspace."""
    b = _b()
    prec = pj._Prec(pj.PJ_BF16, 1, 0, 0)
    M, N, K, Kb, R = 300, 200, 1000, 128, 32
    fwd = lib.proj_gemm_workspace_size(M, N, K, Kb, R, ctypes.byref(b), ctypes.byref(prec))
    bwd = lib.proj_gemm_backward_workspace_size(M, N, K, Kb, R, ctypes.byref(b), ctypes.byref(prec))
    assert fwd > 0 and bwd > 0
    buf = ctypes.c_void_p(1 << 21)                                       # dY, dA, dB: aligned, never dereferenced
    ws_a, ws_b = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 40)   # aligned, never dereferenced

    def call(fws, fbytes, ws):
        return lib.proj_gemm_backward_saved(fws, fbytes, buf, N, buf, K, buf, N, M, N, K, pj.PJ_F32, pj.PJ_F32,
                                            Kb, R, ctypes.byref(b), ctypes.byref(prec), ws, bwd, None)

    assert call(None, fwd, ws_a) == pj.PJ_EINVAL and "fwd_workspace" in pj.last_error()
    assert call(ws_b, fwd - 1, ws_a) == pj.PJ_EINVAL and "fwd_workspace" in pj.last_error()
    assert call(ws_a, fwd, ws_a) == pj.PJ_EINVAL and "different" in pj.last_error()
    split = pj._Prec(pj.PJ_BF16, 2, 0, 0)
    st = lib.proj_gemm_backward_saved(ws_b, fwd, buf, N, buf, K, buf, N, M, N, K, pj.PJ_F32, pj.PJ_F32, Kb, R,
                                      ctypes.byref(b), ctypes.byref(split), ws_a, bwd, None)
    assert st == pj.PJ_EUNSUPPORTED
