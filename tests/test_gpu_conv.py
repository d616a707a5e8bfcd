"""Projected cross-correlation on the GPU against the FP64 oracle and the exact result."""
import numpy as np
import pytest
import torch

import oracle
import paper_1411_2860_gb300 as pj
import synth
from helpers import U_BF16, conv_abs_entries, gamma

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    pj.build()
    assert torch.cuda.is_available()


def conv_bound(s, k, R, mm, tt):
    """Elementwise bound for the box-basis GPU path (BF16 components, FP32 sums)."""
    T = k.shape[1]
    Lb = T // R
    f = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(Lb) * (1 + U_BF16) ** 2 + 2 * gamma(R) * (1 + U_BF16) ** 2
    return f * conv_abs_entries(s, k, R, mm, tt)


def run(s, k, R):
    out = pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), R)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("S,T,nt,R", [(12000, 1024, 64, 1024), (12000, 1024, 64, 256), (12000, 1024, 64, 64),
                                       (9001, 1024, 5, 512), (20000, 4096, 37, 4096), (5000, 128, 64, 128),
                                       (70000, 4096, 64, 64), (60000, 1024, 40, 256), (60000, 1024, 8, 1024),
                                       (30000, 512, 32, 128)])
def test_conv_parity_all_lags(S, T, nt, R):
    """Template counts 40, 8 and 32 cover epilogue warps whose 32 templates are
    partly or wholly past the last one on the TMA-store path."""
    s, k, _ = synth.audio_workload(S, T, nt, seed=3)
    got = run(s, k, R)
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    if (S - T + 1) * T * 64 <= 2e9:
        ref = oracle.conv_proj(s64, k64, R, "haar", 64)
        mm, tt = np.meshgrid(np.arange(S - T + 1), np.arange(nt), indexing="ij")
        mm, tt = mm.ravel(), tt.ravel()
        sel = np.random.default_rng(0).choice(len(mm), size=min(len(mm), 3000), replace=False)
        bound = conv_bound(s64, k64, R, mm[sel], tt[sel])
        assert np.all(np.abs(got.ravel()[sel] - ref.ravel()[sel]) <= bound)
        assert oracle.rel_fro(got, ref) <= 4e-3
    else:
        rng = np.random.default_rng(1)
        mm = rng.integers(0, S - T + 1, 2000)
        tt = rng.integers(0, nt, 2000)
        ref = oracle.conv_proj_entries(s64, k64, mm, tt, R, "haar", 64)
        bound = conv_bound(s64, k64, R, mm, tt)
        assert np.all(np.abs(got[mm, tt] - ref) <= bound)


def test_conv_single_lag_and_one_template():
    s, k, _ = synth.audio_workload(4096, 4096, 1, seed=4)
    got = run(s, k, 1024)
    ref = oracle.conv_proj(s.astype(np.float64), k.astype(np.float64), 1024, "haar", 64)
    assert got.shape == (1, 1)
    assert abs(got[0, 0] - ref[0, 0]) <= conv_bound(s.astype(np.float64), k.astype(np.float64), 1024, [0], [0])[0]


def test_conv_lag_boundaries_exact_tail():
    """Last valid lags of a signal whose lag count is not a multiple of any tile size."""
    s, k, _ = synth.audio_workload(3 * 4096 + 77, 1024, 64, seed=5)
    got = run(s, k, 512)
    lags = s.shape[0] - 1024 + 1
    mm = np.arange(lags - 300, lags)
    tt = np.arange(300) % 64
    ref = oracle.conv_proj_entries(s.astype(np.float64), k.astype(np.float64), mm, tt, 512, "haar", 64)
    assert np.all(np.abs(got[mm, tt] - ref) <= conv_bound(s.astype(np.float64), k.astype(np.float64), 512, mm, tt))


def test_conv_staged_matches_single_call():
    s, k, _ = synth.audio_workload(30000, 1024, 64, seed=6)
    st, kt = torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV)
    r1 = pj.proj_conv(st, kt, 256)
    ws = torch.empty(pj.conv_workspace_size(30000, 1024, 64, 256), dtype=torch.uint8, device=DEV)
    pj.proj_conv_project(st, kt, 256, ws)
    r2 = torch.empty_like(r1)
    pj.proj_conv_correlate(30000, 1024, 64, 256, r2, ws)
    pj.check(ws)
    assert torch.equal(r1, r2)


def test_conv_host_buffers():
    s, k, _ = synth.audio_workload(20000, 1024, 64, seed=7)
    r_host = pj.proj_conv(torch.from_numpy(s).pin_memory(), torch.from_numpy(k).pin_memory(), 1024)
    r_dev = pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), 1024).cpu()
    assert r_host.device.type == "cpu" and torch.equal(r_host, r_dev)


# ------------------------------------------- audio workload at full size --

@pytest.fixture(scope="module")
def audio_full():
    return synth.audio_workload(1 << 20, 4096, 64, seed=0)


@pytest.mark.parametrize("R", [4096, 1024, 256, 64])
def test_audio_full_size_sampled(audio_full, R):
    """S = 2^20, 64 templates of 4096: sampled entries vs the oracle, and the method error."""
    s, k, off = audio_full
    got = run(s, k, R)
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    rng = np.random.default_rng(2)
    mm = np.concatenate([rng.integers(0, s.shape[0] - 4096 + 1, 1500), off])
    tt = np.concatenate([rng.integers(0, 64, 1500), np.arange(64)])
    ref = oracle.conv_proj_entries(s64, k64, mm, tt, R, "haar", 64)
    assert np.all(np.abs(got[mm, tt] - ref) <= conv_bound(s64, k64, R, mm, tt))
    if R == 4096:
        # projected at full R reproduces the exact correlation within BF16 accuracy, below 1e-3 here
        ex = oracle.conv_proj_entries(s64, k64, mm, tt, 4096, "haar", 64)
        assert oracle.rel_fro(got[mm, tt], ex) <= 1e-3
        # every template's true offset is its best match
        assert np.all(np.argmax(got, axis=0) == off)


def test_conv_rejects_bad_arguments_on_gpu():
    s = torch.zeros(5000, device=DEV)
    k = torch.zeros((4, 1000), device=DEV)
    with pytest.raises(pj.ProjError):
        pj.proj_conv(s, k, 1000)


# ------------------------------------------ every step-th lag, interpolated between

def _interp_bound(s64, k64, R, step, mm, tt, lags):
    """Computed lags: the elementwise bound.  Interpolated lags: the weighted bounds
    of the two neighbours plus the FP32 rounding of the interpolation itself."""
    m0 = mm - mm % step
    m1 = np.minimum(m0 + step, lags - 1)
    has1 = m0 + step < lags
    b0 = conv_bound(s64, k64, R, m0, tt)
    b1 = conv_bound(s64, k64, R, m1, tt)
    w1 = np.where(has1, (mm - m0) / step, 0.0)
    return (1 - w1) * b0 + w1 * b1, m0, np.where(has1, m0 + step, m0)


@pytest.mark.parametrize("S,T,nt,R,step", [(12000, 1024, 64, 256, 2), (9001, 1024, 5, 512, 2),
                                            (30000, 512, 32, 128, 4), (60000, 1024, 40, 256, 4),
                                            (5000, 128, 64, 64, 2), (20000, 4096, 16, 2048, 2)])
def test_conv_interp_parity(S, T, nt, R, step):
    s, k, _ = synth.audio_workload(S, T, nt, seed=4)
    sd, kd = torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV)
    got_t = pj.proj_conv(sd, kd, R, step=step)
    full_t = pj.proj_conv(sd, kd, R)
    assert torch.equal(got_t[::step], full_t[::step])      # computed lags are proj_conv's
    got = got_t.double().cpu().numpy()
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    lags = S - T + 1
    rng = np.random.default_rng(2)
    mm = np.concatenate([rng.integers(0, lags, 2500), np.arange(max(0, lags - 2 * step), lags)])
    tt = rng.integers(0, nt, len(mm))
    ref = oracle.conv_proj_interp_entries(s64, k64, mm, tt, R, step, "haar", 64)
    bound, m0, m1 = _interp_bound(s64, k64, R, step, mm, tt, lags)
    ref0 = oracle.conv_proj_entries(s64, k64, m0, tt, R, "haar", 64)
    ref1 = oracle.conv_proj_entries(s64, k64, m1, tt, R, "haar", 64)
    bound = bound + 4 * 2.0 ** -24 * (np.abs(ref0) + np.abs(ref1))
    err = np.abs(got[mm, tt] - ref)
    assert np.all(err <= bound), np.max(err / bound)


def test_conv_interp_audio_2p20_sampled():
    """The 2^20-sample audio workload, R = 1024, half samples."""
    S, T, nt, R = 1 << 20, 4096, 64, 1024
    s, k, _ = synth.audio_workload(S, T, nt, seed=0)
    got = pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), R, step=2)
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    rng = np.random.default_rng(3)
    lags = S - T + 1
    mm = np.concatenate([rng.integers(0, lags, 600), [lags - 1, lags - 2, 0, 1]])
    tt = rng.integers(0, nt, len(mm))
    ref = oracle.conv_proj_interp_entries(s64, k64, mm, tt, R, 2, "haar", 64)
    bound, m0, m1 = _interp_bound(s64, k64, R, 2, mm, tt, lags)
    ref0 = oracle.conv_proj_entries(s64, k64, m0, tt, R, "haar", 64)
    ref1 = oracle.conv_proj_entries(s64, k64, m1, tt, R, "haar", 64)
    bound = bound + 4 * 2.0 ** -24 * (np.abs(ref0) + np.abs(ref1))
    g = got[torch.from_numpy(mm).to(DEV), torch.from_numpy(tt).to(DEV)].double().cpu().numpy()
    assert np.all(np.abs(g - ref) <= bound)


@pytest.mark.parametrize("R,step", [(4096, 2), (1024, 3), (1024, 8)])
def test_conv_interp_rejects_bad_steps(R, step):
    s, k, _ = synth.audio_workload(20000, 4096, 2, seed=5)
    with pytest.raises(pj.ProjError):
        pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), R, step=step)


@pytest.mark.parametrize("S,T,nt,R,chunks", [(60000, 1024, 40, 256, 4), (20000, 4096, 16, 4096, 3),
                                              (9001, 1024, 5, 512, 1), (30000, 512, 32, 128, 7)])
def test_conv_host_buffers_chunked(S, T, nt, R, chunks):
    """proj_conv_host: host signal, templates and output, lags in chunks whose copies
    overlap the next chunk's correlation; every lag equals proj_conv's on the device."""
    s, k, _ = synth.audio_workload(S, T, nt, seed=6)
    sh = torch.from_numpy(s).pin_memory()
    kh = torch.from_numpy(k).pin_memory()
    got = pj.proj_conv_host(sh, kh, R, chunks=chunks)
    dev = pj.proj_conv(sh.to(DEV), kh.to(DEV), R).cpu()
    assert got.device.type == "cpu"
    assert torch.equal(got, dev)
    got2 = pj.proj_conv(sh, kh, R)            # the host path of proj_conv goes through it too
    assert torch.equal(got2, dev)


def conv_general_bound(s, k, R, kind, L, user_C, mm, tt):
    """Elementwise bound of the general-basis path: with |sc_p[x]| <= sum_i |s[x+i]| |c[i,p]|
    and |kd_t[g,p]| <= sum_i |d[p,i]| |k_t[gL+i]| (BF16 components, FP32 sums of L and of R
    terms), |r_gpu - r_R| <= [2u + u^2 + 2 gamma_L (1+u)^2 + 2 gamma_R (1+u)^2]
    * sum_{g,p} |sc_p[m+gL]| |kd_t[g,p]|."""
    C, D = oracle.basis(kind, L, user_C) if user_C is not None else oracle.basis(kind, L)
    T = k.shape[1]
    lp1 = R * L // T
    G = T // L
    Ca, Da = np.abs(C[:, :lp1]), np.abs(D[:lp1, :])
    a = np.abs(s)
    n = len(s) - L + 1
    sc = np.stack([np.convolve(a, Ca[::-1, q], mode="valid")[:n] for q in range(lp1)], axis=1)  # n x lp1
    kd = np.einsum("pi,tgi->tgp", Da, np.abs(k).reshape(k.shape[0], G, L))                      # nt x G x lp1
    out = np.empty(len(mm))
    for e, (m, t) in enumerate(zip(mm, tt)):
        out[e] = np.sum(sc[m + L * np.arange(G)] * kd[t])
    f = 2 * U_BF16 + U_BF16 ** 2 + 2 * gamma(L) * (1 + U_BF16) ** 2 + 2 * gamma(R) * (1 + U_BF16) ** 2
    return f * out


@pytest.mark.parametrize("S,T,nt,kind,L,R", [
    (12000, 1024, 64, "dct2", 8, 1024),   # l+1 = 8: one component group per position, no copies
    (12000, 1024, 64, "dct2", 8, 512),    # l+1 = 4: two shifted copies
    (9001, 1024, 5, "dct2", 8, 256),      # l+1 = 2: four copies
    (20000, 1024, 37, "dct2", 8, 128),    # l+1 = 1: eight copies
    (8000, 200, 16, "dct2", 8, 200),      # T not a multiple of 64: the last template chunk is padded
    (8000, 136, 64, "dct2", 8, 34),       # 17 groups, R = 34
    (10000, 512, 8, "user", 8, 256),      # oblique user basis
    (10000, 1024, 64, "dct2", 16, 1024),  # L = 16, l+1 = 16: four row offsets
    (6000, 640, 3, "dct2", 64, 640),      # L = 64, l+1 = 64: one row offset
])
def test_conv_general_basis_parity(S, T, nt, kind, L, R):
    """Any basis through the general path (phases phi < L, l+1 components per position)
    against the oracle's Eq. 11-13, every lag of a sample of outputs checked elementwise."""
    s, k, _ = synth.audio_workload(S, T, nt, seed=8)
    U = np.eye(L) + 0.25 * np.random.default_rng(L).normal(size=(L, L)) if kind == "user" else None
    got = pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), R, kind, L,
                       user_C=U).double().cpu().numpy()
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    rng = np.random.default_rng(2)
    lags = S - T + 1
    mm = np.concatenate([rng.integers(0, lags, 1500), np.arange(max(0, lags - 100), lags)])
    tt = rng.integers(0, nt, len(mm))
    ref = oracle.conv_proj_entries(s64, k64, mm, tt, R, kind, L, U)
    bound = conv_general_bound(s64, k64, R, kind, L, U, mm, tt)
    assert np.all(np.abs(got[mm, tt] - ref) <= bound), np.max(np.abs(got[mm, tt] - ref) / bound)


def test_conv_general_basis_full_matches_oracle_and_exact():
    """DCT-II at full R (l+1 = L): the whole correlation against the oracle, and the
    truncation-free result against the exact correlation to BF16 accuracy."""
    S, T, nt = 9000, 512, 24
    s, k, _ = synth.audio_workload(S, T, nt, seed=9)
    got = pj.proj_conv(torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV), T, "dct2", 8).double().cpu().numpy()
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    ref = oracle.conv_proj(s64, k64, T, "dct2", 8)
    assert oracle.rel_fro(got, ref) <= 4e-3
    assert oracle.rel_fro(got, oracle.conv_exact(s64, k64)) <= 4e-3


def test_conv_general_basis_half_samples_and_host_buffers():
    """Every other lag computed with the DCT (phases of L = 8) and the rest interpolated;
    the host-buffer entry point gives the device result bit for bit."""
    S, T, nt, R = 20000, 1024, 16, 512
    s, k, _ = synth.audio_workload(S, T, nt, seed=10)
    sd, kd = torch.from_numpy(s).to(DEV), torch.from_numpy(k).to(DEV)
    full = pj.proj_conv(sd, kd, R, "dct2", 8)
    half = pj.proj_conv(sd, kd, R, "dct2", 8, step=2)
    torch.cuda.synchronize()
    assert torch.equal(full[0::2], half[0::2])
    f, h = full.double().cpu().numpy(), half.double().cpu().numpy()
    mid = 0.5 * (f[0:-2:2] + f[2::2])
    assert np.all(np.abs(h[1:-1:2] - mid) <= 4 * 2.0 ** -24 * (np.abs(f[0:-2:2]) + np.abs(f[2::2])))
    host = pj.proj_conv(torch.from_numpy(s), torch.from_numpy(k), R, "dct2", 8)
    assert torch.equal(host, full.cpu())


@pytest.mark.parametrize("S,T,nt,R", [(30000, 1024, 4, 256), (12000, 4096, 2, 4096)])
def test_conv_e4m3_single_call_matches_the_batch_and_the_oracle(S, T, nt, R):
    """proj_conv with E4M3 components (one lowered instance on the block-scaled MMA):
    within the E4M3 bound of the oracle and equal to the same correlation run as a
    batch entry."""
    from test_gpu_batch import _check_conv_e4m3
    s, k, _ = synth.audio_workload(S, T, nt, seed=S + R)
    sd = torch.from_numpy(s).to(DEV)
    kd = torch.from_numpy(k).to(DEV)
    out = pj.proj_conv(sd, kd, R, compute="e4m3")
    torch.cuda.synchronize()
    _check_conv_e4m3(dict(s=sd, k=kd, out=out, R=R), n=800, seed=R)
    out2 = torch.full_like(out, float("nan"))
    plan = pj.BatchPlan([pj.batch_conv(sd, kd, out2, R, compute="e4m3")])
    plan.run()
    plan.check()
    assert torch.equal(out, out2)
