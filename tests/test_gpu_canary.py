"""Guard regions around every output: a kernel that writes outside its output
(a ragged tile's tail, a pair's stand-in tile, a stream-K reduction, a TMA box
past the edge) changes a canary.  The outputs live inside larger buffers filled
with a sentinel; after each call everything outside the output view must still
hold the sentinel bit for bit, and the output itself must hold no sentinel."""
import numpy as np
import pytest
import torch

import paper_1411_2860_gb300 as pj
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
SENTINEL = -12345.678


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def _guarded(rows, cols, dtype, pad_rows=3, pad_cols=5):
    """A view of rows x cols inside a sentinel-filled buffer; the view starts 16-byte
    aligned and its row pitch is a multiple of 16 bytes."""
    es = torch.empty((), dtype=dtype).element_size()
    per16 = 16 // es
    pitch = -(-(cols + pad_cols) // per16) * per16
    big = torch.full((rows + 2 * pad_rows, pitch), SENTINEL, dtype=dtype, device=DEV)
    col0 = per16  # 16-byte aligned start inside each row
    if col0 + cols > pitch:
        big = torch.full((rows + 2 * pad_rows, pitch + per16), SENTINEL, dtype=dtype, device=DEV)
    view = big[pad_rows:pad_rows + rows, col0:col0 + cols]
    return big, view, (slice(pad_rows, pad_rows + rows), slice(col0, col0 + cols))


def _check_guards(big, region):
    mask = torch.ones_like(big, dtype=torch.bool)
    mask[region] = False
    sentinel = torch.tensor(SENTINEL, dtype=big.dtype, device=DEV)
    bad = mask & (big != sentinel)
    if torch.any(bad):
        idx = torch.nonzero(bad)[:8].tolist()
        vals = [float(big[r, c]) for r, c in idx]
        raise AssertionError(f"a kernel wrote outside its output (region {region}, buffer {tuple(big.shape)}): "
                             f"{int(bad.sum())} elements, first at {idx} = {vals}")
    assert not torch.any(big[region] == sentinel), "an output element was not written"


@pytest.mark.parametrize("M,N,K,Kb,R,split,out_dtype", [
    (300, 200, 1000, 128, 32, 1, torch.float32),     # even tile columns: CTA pairs
    (513, 257, 777, 64, 16, 2, torch.float32),       # odd tile columns, ragged everything
    (300, 260, 20000, 128, 128, 2, torch.float32),   # stream-K (partial products added into the output)
    (129, 384, 2048, 256, 256, 1, torch.bfloat16),   # BF16 output
    (1, 1, 8, 8, 8, 1, torch.float32),
])
def test_gemm_writes_only_its_output(M, N, K, Kb, R, split, out_dtype):
    rng = np.random.default_rng(M + N)
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    big, Y, region = _guarded(M, N, out_dtype)
    pj.proj_gemm(A, B, Kb, R, split=split, out=Y)
    torch.cuda.synchronize()
    _check_guards(big, region)


def test_e4m3_gemm_writes_only_its_output():
    rng = np.random.default_rng(9)
    M, N, K = 260, 256, 1536
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    big, Y, region = _guarded(M, N, torch.float32)
    pj.proj_gemm(A, B, 128, 128, compute="e4m3", split=2, out=Y)
    torch.cuda.synchronize()
    _check_guards(big, region)


@pytest.mark.parametrize("S,T,nt,R,step", [(12000, 1024, 64, 1024, 1), (9001, 1024, 5, 256, 1),
                                            (30000, 512, 37, 128, 1), (20000, 1024, 40, 256, 1),
                                            (20001, 1024, 40, 256, 2), (9001, 1024, 5, 256, 4)])
def test_conv_writes_only_its_output(S, T, nt, R, step):
    """nt = 40: the last 32-template box of the TMA-store epilogue is partly past the
    templates; step > 1: the interpolated lags are written by their own kernel."""
    s, k, _ = synth.audio_workload(S, T, nt, seed=7)
    lags = S - T + 1
    guard = 1024
    flat = torch.full((lags * nt + 2 * guard,), SENTINEL, dtype=torch.float32, device=DEV)
    out = flat[guard:guard + lags * nt].view(lags, nt)
    pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), R, out=out, step=step)
    torch.cuda.synchronize()
    sentinel = torch.tensor(SENTINEL, device=DEV)
    assert torch.equal(flat[:guard], sentinel.expand(guard)) and torch.equal(flat[-guard:], sentinel.expand(guard))
    assert not torch.any(out == sentinel)


@pytest.mark.parametrize("tuning", [None, {"solo": 1}])
def test_batch_writes_only_its_outputs(tuning):
    rng = np.random.default_rng(11)
    shapes = [(300, 200, 1000), (100, 513, 2560), (37, 130, 700), (256, 256, 4096)]
    guards, descs = [], []
    for M, N, K in shapes:
        A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
        B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
        big, Y, region = _guarded(M, N, torch.float32)
        guards.append((big, region, A, B))
        descs.append(pj.batch_gemm(A, B, Y, 128, 64, split=2))
    plan = pj.BatchPlan(descs, tuning=tuning)
    plan.run()
    plan.check()
    for big, region, _, _ in guards:
        _check_guards(big, region)


@pytest.mark.parametrize("M,N,K,Kb,R", [(130, 90, 515, 128, 32), (64, 257, 1024, 256, 64)])
def test_backward_writes_only_its_outputs(M, N, K, Kb, R):
    rng = np.random.default_rng(M)
    A = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(rng.normal(size=(K, N)).astype(np.float32)).to(DEV)
    dY = torch.from_numpy(rng.normal(size=(M, N)).astype(np.float32)).to(DEV)
    bigA, dA, regA = _guarded(M, K, torch.float32)
    bigB, dB, regB = _guarded(K, N, torch.float32)
    pj.proj_gemm_backward(A, B, dY, Kb, R, dA=dA, dB=dB)
    torch.cuda.synchronize()
    _check_guards(bigA, regA)
    _check_guards(bigB, regB)


def test_batch_correlation_writes_only_its_output():
    s, k, _ = synth.audio_workload(20000, 1024, 1, seed=12)
    lags = 20000 - 1024 + 1
    guard = 1024
    flat = torch.full((lags + 2 * guard,), SENTINEL, dtype=torch.float32, device=DEV)
    out = flat[guard:guard + lags].view(lags, 1)
    plan = pj.BatchPlan([pj.batch_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), out, 256)])
    plan.run()
    plan.check()
    sentinel = torch.tensor(SENTINEL, device=DEV)
    assert torch.equal(flat[:guard], sentinel.expand(guard)) and torch.equal(flat[-guard:], sentinel.expand(guard))
    assert not torch.any(out == sentinel)
