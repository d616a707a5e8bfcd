"""Benchmark of the projected GEMM / CONV hot path on GB300.

Default workload (``--workload conv``): one audio-like signal of 2^20 samples
(32 tones in 50-8000 Hz at 44.1 kHz plus noise at 20 dB SNR) correlated with 64
templates of 4096 samples cut from it, Haar projection (L = 64), R = 4096
components per template -- the setting whose error against the FP64 exact
correlation stays below 1e-3.  A step is one pass of the whole path: project
signal and templates, then the reduced correlation at all 1,044,481 lags.
Metric: effective TFLOP/s = 2 * lags * templates * T / time (full T, whatever R).

Other workloads (reported, not the headline): ``face-gemm`` (4096 x 10304 by
10304 x 2048, block 512) and ``layer`` (forward + backward of X 8192x4096 times
W 4096x4096 in BF16, block 256, R = 64).  Effective TFLOP/s = 2 M N K / t.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload conv|face-gemm|layer] [--R R] [--split S]

Timed steps are CUDA-graph replays of the library calls, bracketed by CUDA
events on the launching stream, with L2 flushed (256 MiB write) between steps
outside the events.  Under torchrun each rank runs its own independent
instance (weak scaling, no data-path collective); the timed region is
bracketed by barriers and the maximum over ranks is reported.
--impl reference times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

S, T, NT, L = 1 << 20, 4096, 64, 64
LAGS = S - T + 1
EFF_FLOPS = 2.0 * LAGS * NT * T           # effective work of one CONV step (full T)
METRIC = "effective TFLOP/s (2MNK/t) projected vs exact GEMM/CONV on GB300 at rel. err ≤1e-3"

# DRAM traffic of one conv_tc_kernel launch at R = 4096 from ncu, recorded with the
# hash of the kernel source it was measured on (null once the source changes).
TRAFFIC = {"sha256": "167a4666747144d233bc43fa359aa9db6ad9dec96d7f9cb97e4183640f3f7568",
           "bytes": 17988352 + 206045184}   # profiles/conv_tc_audio_2p20x64x4096_R4096.md


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


def source_hash(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sms, maxes, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxes.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxes) if maxes else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sms)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device) -> float:
    """Maximum of x over all ranks (identity when world == 1)."""
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, max_ms: float, flops_per_step: float = EFF_FLOPS) -> float:
    """Whole-job TFLOP/s: every rank runs `steps` independent steps; time = slowest rank."""
    return world * flops_per_step * steps / (max_ms * 1e-3) / 1e12


def sampled_rel_err(sig, tpl, out, n=1024, seed=11, transposed=False):
    """Relative error of sampled CONV outputs against the exact correlation (float64 on the GPU)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    nl = out.shape[1] if transposed else out.shape[0]
    nt = out.shape[0] if transposed else out.shape[1]
    mm = torch.randint(0, nl, (n,), generator=g).to(sig.device)
    tt = torch.randint(0, nt, (n,), generator=g).to(sig.device)
    idx = mm[:, None] + torch.arange(tpl.shape[1], device=sig.device)[None, :]
    exact = (sig.double()[idx] * tpl.double()[tt]).sum(dim=1)
    got = (out[tt, mm] if transposed else out[mm, tt]).double()
    return float(torch.linalg.norm(got - exact) / torch.linalg.norm(exact))


def sampled_rel_err_gemm(A, B, Y, n=1024, seed=12):
    """Relative error of sampled GEMM outputs against the exact product (float64 on the GPU)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    ii = torch.randint(0, Y.shape[0], (n,), generator=g).to(A.device)
    jj = torch.randint(0, Y.shape[1], (n,), generator=g).to(A.device)
    exact = (A[ii].double() * B[:, jj].t().double()).sum(dim=1)
    got = Y[ii, jj].double()
    return float(torch.linalg.norm(got - exact) / torch.linalg.norm(exact))


def capture(fn, stream):
    """CUDA graph of the library calls made by fn on `stream`."""
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
        fn()
    return g


class _Direct:
    """Stand-in for a graph: replay() calls the library directly."""

    def __init__(self, fn):
        self.replay = fn


def time_graphs(graphs, steps, flush, stream):
    """Per-step device times (ms) of a sequence of graphs; returns per-graph lists and the step total."""
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(graphs) + 1)] for _ in range(steps)]
    torch.cuda.synchronize()
    for ev in evs:
        flush.zero_()                    # evict L2 between timed steps (outside the events)
        ev[0].record(stream)
        for g, e in zip(graphs, ev[1:]):
            g.replay()
            e.record(stream)
    torch.cuda.synchronize()
    parts = [[ev[i].elapsed_time(ev[i + 1]) for ev in evs] for i in range(len(graphs))]
    total = sum(ev[0].elapsed_time(ev[-1]) for ev in evs)
    return parts, total


def median_ms(fn, stream, flush, reps=5):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


# ----------------------------------------------------------------- CONV --

def conv_exact_baselines(sig, tpl, stream, flush):
    """cuDNN conv1d (cross-correlation) on the same workload in FP32, TF32 and BF16."""
    import torch.nn.functional as F
    res = []
    torch.backends.cudnn.benchmark = True
    x = sig.view(1, 1, -1)
    w = tpl.view(tpl.shape[0], 1, -1)
    for name, dt, tf32 in (("cudnn conv1d fp32", torch.float32, False), ("cudnn conv1d tf32", torch.float32, True),
                           ("cudnn conv1d bf16", torch.bfloat16, False)):
        torch.backends.cudnn.allow_tf32 = tf32
        xx, ww = x.to(dt), w.to(dt)
        try:
            ms = median_ms(lambda: F.conv1d(xx, ww), stream, flush, reps=3)
            out = F.conv1d(xx, ww)[0].float()
            err = sampled_rel_err(sig, tpl, out, transposed=True)
            del out
            res.append({"impl": name, "ms": round(ms, 4), "value": round(EFF_FLOPS / (ms * 1e-3) / 1e12, 2),
                        "rel_err_vs_exact": err})
        except RuntimeError as e:     # cuDNN may refuse a configuration
            res.append({"impl": name, "error": str(e)[:120]})
        torch.cuda.empty_cache()
    torch.backends.cudnn.allow_tf32 = False
    return res


def run_conv(args, pj, world, rank, dev, stream, flush):
    import synth
    R = args.R
    s_np, k_np, _ = synth.audio_workload(S, T, NT, seed=rank)
    sig = torch.from_numpy(s_np).to(dev)
    tpl = torch.from_numpy(k_np).to(dev)
    out = torch.empty((LAGS, NT), dtype=torch.float32, device=dev)
    cb, cL = args.conv_basis, args.conv_L
    ws = torch.empty(pj.conv_workspace_size(S, T, NT, R, cb, cL), dtype=torch.uint8, device=dev)

    def project():
        pj.proj_conv_project(sig, tpl, R, ws, cb, cL, stream=torch.cuda.current_stream())

    def correlate():
        pj.proj_conv_correlate(S, T, NT, R, out, ws, cb, cL, stream=torch.cuda.current_stream())

    # nvidia-smi samples every 100 ms from here to the end of the timed region
    # (it takes a moment to start, so it is started before the warm-up).
    clocks = ClockSampler(dev.index)
    clocks.start()
    for _ in range(args.warmup):
        project()
        correlate()
    torch.cuda.synchronize()
    pj.check(ws)
    if args.no_graph:
        stages = [_Direct(project), _Direct(correlate)]
    else:
        stages = [capture(project, stream), capture(correlate, stream)]
        for g in stages:
            g.replay()
    if world > 1:
        torch.distributed.barrier()
    (proj_ms, kern_ms), step_ms = time_graphs(stages, args.steps, flush, stream)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    pj.check(ws)
    total_ms = reduce_max(step_ms, world, dev)
    rel_err = sampled_rel_err(sig, tpl, out)

    # end to end through the public API with host buffers (pinned), copies inside the region
    # (proj_conv_host: the lags in chunks, each chunk's copy to the host overlapping the next's correlation)
    s_host = torch.from_numpy(s_np).pin_memory()
    k_host = torch.from_numpy(k_np).pin_memory()
    r_host = torch.empty((LAGS, NT), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 20))
    e2e_chunks = 8
    ws_host = torch.empty(pj.conv_host_workspace_size(S, T, NT, R, chunks=e2e_chunks), dtype=torch.uint8, device=dev)
    pj.proj_conv_host(s_host, k_host, R, out=r_host, workspace=ws_host, chunks=e2e_chunks, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pj.proj_conv_host(s_host, k_host, R, out=r_host, workspace=ws_host, chunks=e2e_chunks, stream=stream)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
    e2e_sweep = []
    if rank == 0 and not args.no_sweep:
        for ch in (1, 2, 4):
            wsc = torch.empty(pj.conv_host_workspace_size(S, T, NT, R, chunks=ch), dtype=torch.uint8, device=dev)
            pj.proj_conv_host(s_host, k_host, R, out=r_host, workspace=wsc, chunks=ch, stream=stream)
            t1 = time.perf_counter()
            for _ in range(e2e_steps):
                pj.proj_conv_host(s_host, k_host, R, out=r_host, workspace=wsc, chunks=ch, stream=stream)
            dt = (time.perf_counter() - t1) / e2e_steps
            e2e_sweep.append({"chunks": ch, "ms": round(dt * 1e3, 4), "value": round(EFF_FLOPS / dt / 1e12, 2)})
            del wsc
        e2e_sweep.append({"chunks": e2e_chunks, "ms": round(e2e_s / e2e_steps * 1e3, 4),
                          "value": round(EFF_FLOPS / (e2e_s / e2e_steps) / 1e12, 2)})
    del ws_host

    extra = {}
    if rank == 0 and not args.no_sweep:
        sweep = []
        # the Haar box path at every R, and the general path with the DCT-II (L = 8) beside it
        for Rs, sb, sL in ((4096, "haar", 64), (1024, "haar", 64), (256, "haar", 64), (64, "haar", 64),
                           (4096, "dct2", 8), (2048, "dct2", 8), (1024, "dct2", 8), (512, "dct2", 8)):
            ws2 = torch.empty(pj.conv_workspace_size(S, T, NT, Rs, sb, sL), dtype=torch.uint8, device=dev)
            out2 = torch.empty_like(out)

            def p2():
                pj.proj_conv_project(sig, tpl, Rs, ws2, sb, sL, stream=torch.cuda.current_stream())

            def c2():
                pj.proj_conv_correlate(S, T, NT, Rs, out2, ws2, sb, sL, stream=torch.cuda.current_stream())

            p2()
            c2()
            gs = [_Direct(p2), _Direct(c2)] if args.no_graph else [capture(p2, stream), capture(c2, stream)]
            (pm, cm), tot = time_graphs(gs, 10, flush, stream)
            ms = tot / 10
            cmed = statistics.median(cm)
            sweep.append({"R": Rs, "basis": sb, "L": sL, "ms": round(ms, 4),
                          "value": round(EFF_FLOPS / (ms * 1e-3) / 1e12, 2),
                          "project_ms": round(statistics.median(pm), 4), "correlate_ms": round(cmed, 4),
                          "correlate_tflops_reduced": round(2.0 * LAGS * NT * Rs / (cmed * 1e-3) / 1e12, 1),
                          "correlate_out_gbs": round(LAGS * NT * 4 / (cmed * 1e-3) / 1e9, 1),
                          "rel_err_vs_exact": sampled_rel_err(sig, tpl, out2)})
            del ws2, out2, gs
        extra["r_sweep"] = sweep
        # every other lag computed, the rest interpolated (the paper's half-sample option)
        half = []
        for Rs in (2048, 1024, 256):
            ws2 = torch.empty(pj.conv_workspace_size(S, T, NT, Rs), dtype=torch.uint8, device=dev)
            out2 = torch.empty_like(out)
            for stp in (1, 2):
                def f2():
                    pj.proj_conv(sig, tpl, Rs, out=out2, workspace=ws2, stream=torch.cuda.current_stream(), step=stp)

                f2()
                g2 = _Direct(f2) if args.no_graph else capture(f2, stream)
                (tm,), tot = time_graphs([g2], 10, flush, stream)
                ms = tot / 10
                half.append({"R": Rs, "step": stp, "ms": round(ms, 4),
                             "value": round(EFF_FLOPS / (ms * 1e-3) / 1e12, 2),
                             "rel_err_vs_exact": sampled_rel_err(sig, tpl, out2)})
                del g2
            del ws2, out2
        extra["half_samples"] = half
        if not args.no_exact:
            extra["exact_baselines"] = conv_exact_baselines(sig, tpl, stream, flush)
    if rank != 0:
        return None
    hbm, bf16_burst, _, src = peaks()
    kern = statistics.mean(kern_ms)
    tensor_bound = R >= 1024
    tflops = 2.0 * LAGS * NT * R / (kern * 1e-3) / 1e12
    gbs = LAGS * NT * 4 / (kern * 1e-3) / 1e9
    traffic = TRAFFIC["bytes"] if TRAFFIC["sha256"] == source_hash(
        "paper_1411_2860_gb300/csrc/conv_tc.cu") and R == 4096 else None
    line = {
        "metric": METRIC, "value": round(job_throughput(world, args.steps, total_ms), 3), "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"projected cross-correlation: audio-like signal 2^20 samples x 64 templates "
                               f"of 4096, {'Haar' if cb == 'haar' else cb} L={cL}, R={R}, all {LAGS} lags",
                   "S": S, "T": T, "n_templates": NT, "R": R, "basis": cb, "L": cL,
                   "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                   "timing": "direct library calls" if args.no_graph
                   else "CUDA graph replay of the two library stages",
                   "parallelism": f"independent instance per GPU x{world}"},
        "rel_err_sampled_vs_exact": rel_err,
        "roofline": {"bound": "tensor" if tensor_bound else "hbm",
                     "achieved": round(tflops if tensor_bound else gbs, 2),
                     "peak": bf16_burst if tensor_bound else hbm,
                     "unit": "TFLOP/s" if tensor_bound else "GB/s",
                     "frac": round((tflops / bf16_burst) if tensor_bound else (gbs / hbm), 4),
                     "traffic": traffic, "kernel": "conv_tc_kernel", "kernel_ms": round(kern, 4),
                     "peak_source": f"{src}: MEASURED_PEAKS.json "
                                    + ("bf16 dense burst" if tensor_bound else "hbm copy")},
        "stage_ms": {"project": round(statistics.mean(proj_ms), 4), "correlate": round(kern, 4)},
        "e2e": {"value": round(job_throughput(world, e2e_steps, e2e_s * 1e3), 3), "unit": "TFLOP/s",
                "h2d_bytes_per_step": (S + NT * T) * 4, "d2h_bytes_per_step": LAGS * NT * 4,
                "api": f"proj_conv_host, {e2e_chunks} lag chunks", "chunk_sweep": e2e_sweep},
        "gpu_launches": 2 * args.steps,   # conv_project_kernel + conv_tc_kernel per step (the L2 flush is torch's)
        "clocks": clk,
    }
    line.update(extra)
    return line


# ----------------------------------------------------------------- GEMM --

def gemm_exact_baselines(A, B, stream, flush):
    res = []
    for name, dt, tf32 in (("cublas fp32", torch.float32, False), ("cublas tf32", torch.float32, True),
                           ("cublas bf16", torch.bfloat16, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        Ab, Bb = A.to(dt), B.to(dt)
        ms = median_ms(lambda: torch.matmul(Ab, Bb), stream, flush)
        Y = torch.matmul(Ab, Bb).float()
        res.append({"impl": name, "ms": round(ms, 4),
                    "value": round(2.0 * A.shape[0] * B.shape[1] * A.shape[1] / (ms * 1e-3) / 1e12, 2),
                    "rel_err_vs_exact": sampled_rel_err_gemm(A, B, Y)})
        del Ab, Bb, Y
    torch.backends.cuda.matmul.allow_tf32 = False
    return res


def run_face_gemm(args, pj, world, rank, dev, stream, flush):
    import synth
    M, K, N, Kb = 4096, 10304, 2048, 512
    A = torch.from_numpy(synth.face_probes(M, seed=0)).to(dev)
    B = torch.from_numpy(synth.orthonormal_features(K, N, seed=1)).to(dev)
    eff = 2.0 * M * N * K
    rows = []
    computes = ["bf16", "e4m3"] if args.compute is None else [args.compute]
    settings = [(R, sp, c, 0) for c in computes for R, sp in ((512, 2), (512, 1), (128, 1), (64, 1))] \
        if args.R is None else [(args.R, args.split, c, args.split_lead) for c in computes]
    settings = [s + ("dct2",) for s in settings]
    if args.R is None and "bf16" in computes:
        # precision tiering: the lo term only on the low-order projections
        settings += [(512, 2, "bf16", lead, "dct2") for lead in (1, 2, 4)]
        # a basis learned from the probes (principal axes of their 8-sample groups)
        settings += [(R_, 1, "bf16", 0, "pca") for R_ in (128, 64)]
    groups = A.double().reshape(-1, 8)
    # the 8 x 8 second-moment matrix on the GPU, its eigenvectors on the host
    pca_C = np.linalg.eigh((groups.T @ groups / groups.shape[0]).cpu().numpy())[1][:, ::-1].copy()
    # ||A B||_F in FP64, to state the a-posteriori bounds of proj_gemm_report relative to it
    ynorm = float(torch.linalg.matrix_norm(A.double() @ B.double()))
    for R, split, compute, lead, basis in settings:
        uc = pca_C if basis == "pca" else None
        bk = "user" if basis == "pca" else "dct2"
        ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R, bk, compute=compute, split=split, split_lead=lead,
                                                user_C=uc), dtype=torch.uint8, device=dev)
        Y = torch.empty((M, N), dtype=torch.float32, device=dev)

        if args.fused:   # the feature matrix projected once; the probes inside the GEMM
            pj.proj_gemm_project(None, B, Kb, R, ws, bk, compute=compute, split=split, M=M, N=N, K=K,
                                 split_lead=lead, user_C=uc)

        def gp_fn():
            if not args.fused:
                pj.proj_gemm_project(A, B, Kb, R, ws, bk, compute=compute, split=split,
                                     stream=torch.cuda.current_stream(), split_lead=lead, user_C=uc)

        def gm_fn():
            if args.fused:
                pj.proj_gemm_fused(A, Y, Kb, R, ws, bk, split=split, user_C=uc, stream=torch.cuda.current_stream())
            else:
                pj.proj_gemm_multiply(Y, K, Kb, R, ws, bk, compute=compute, split=split,
                                      stream=torch.cuda.current_stream(), split_lead=lead, user_C=uc)

        gp_fn()
        gm_fn()
        gs = [_Direct(gp_fn), _Direct(gm_fn)] if args.no_graph else [capture(gp_fn, stream), capture(gm_fn, stream)]
        for _ in range(args.warmup):
            for g in gs:
                g.replay()
        (pm, mm), tot = time_graphs(gs, args.steps, flush, stream)
        pj.check(ws)
        ms = tot / args.steps
        kp = R * (K // Kb) + (R // (Kb // 8)) * ((K % Kb) // 8)
        kt = kp // (R // (Kb // 8)) * lead if lead else kp
        red = 2.0 * M * N * (kp + (2 * kt if split == 2 else 0))
        mmed = statistics.median(mm)
        rep = pj.proj_gemm_report(A, B, Kb, R, bk, compute=compute, split=split, split_lead=lead, user_C=uc)
        rows.append({"R": R, "split": split, "split_lead": lead, "compute": compute, "basis": basis,
                     "ms": round(ms, 4),
                     "value": round(eff / (ms * 1e-3) / 1e12, 2),
                     "project_ms": round(statistics.median(pm), 4), "multiply_ms": round(mmed, 4),
                     "multiply_tflops_reduced": round(red / (mmed * 1e-3) / 1e12, 1),
                     "rel_err_vs_exact": sampled_rel_err_gemm(A, B, Y),
                     # a-posteriori truncation bound (proj_gemm_report) over ||A B||_F; None for a user basis
                     "trunc_bound_rel": rep["trunc_bound"] / ynorm if rep["trunc_bound"] >= 0 else None})
        del ws, Y, gs
    # pre-projected operand cache: B (the feature matrix) projected once, each new
    # batch of probes projected alone and multiplied with the cached B_d
    cached = []
    if args.R is None:
        for R, split, lead in ((512, 2, 0), (512, 2, 1), (512, 1, 0), (128, 1, 0), (64, 1, 0)):
            ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R, split=split, split_lead=lead), dtype=torch.uint8,
                             device=dev)
            Y = torch.empty((M, N), dtype=torch.float32, device=dev)
            pj.proj_gemm_project(None, B, Kb, R, ws, split=split, M=M, N=N, K=K, split_lead=lead)

            def step_fn():
                pj.proj_gemm_project(A, None, Kb, R, ws, split=split, N=N, split_lead=lead,
                                     stream=torch.cuda.current_stream())
                pj.proj_gemm_multiply(Y, K, Kb, R, ws, split=split, split_lead=lead, stream=torch.cuda.current_stream())

            step_fn()
            g = _Direct(step_fn) if args.no_graph else capture(step_fn, stream)
            for _ in range(args.warmup):
                g.replay()
            (tm,), tot = time_graphs([g], args.steps, flush, stream)
            ms = tot / args.steps
            cached.append({"R": R, "split": split, "split_lead": lead, "ms": round(ms, 4),
                           "value": round(eff / (ms * 1e-3) / 1e12, 2),
                           "rel_err_vs_exact": sampled_rel_err_gemm(A, B, Y)})
            del ws, Y, g
    base = gemm_exact_baselines(A, B, stream, flush) if not args.no_exact else []
    return {"workload": "face-gemm 4096x10304 by 10304x2048, block 512, DCT-II L=8", "rows": rows,
            "cached_features": cached,
            "exact_baselines": base}


def run_fp64(args, pj, world, rank, dev, stream, flush):
    """Config 1: FP64 projected GEMM, A 256x512 by B 512x256 (uniform [-1, 1)), block 128,
    DCT-II L = 8: time per call and relative error against the FP64 product at each R."""
    import synth
    A_np, B_np = synth.uniform_pair(256, 512, 256, seed=0)
    A = torch.from_numpy(A_np).to(dev)
    B = torch.from_numpy(B_np).to(dev)
    exact = A @ B
    rows = []
    for R in (128, 64, 32, 16):
        Y = torch.empty((256, 256), dtype=torch.float64, device=dev)
        ws = torch.empty(pj.gemm_workspace_size(256, 256, 512, 128, R, compute="f64"), dtype=torch.uint8,
                         device=dev)

        def fn():
            pj.proj_gemm(A, B, 128, R, compute="f64", out=Y, workspace=ws, stream=torch.cuda.current_stream())

        fn()
        g = _Direct(fn) if args.no_graph else capture(fn, stream)
        for _ in range(args.warmup):
            g.replay()
        (t,), _ = time_graphs([g], max(10, min(args.steps, 200)), flush, stream)
        ms = statistics.median(t)
        rel = float(torch.linalg.norm(Y - exact) / torch.linalg.norm(exact))
        rows.append({"R": R, "ms": round(ms, 4), "reduced_gflop": round(2.0 * 256 * 256 * 512 * R / 128 / 1e9, 4),
                     "rel_err_vs_exact_fp64": rel})
    return {"workload": "fp64 GEMM 256x512 by 512x256, uniform[-1,1), block 128, DCT-II L=8", "rows": rows,
            "note": "the full-R error is rounding only (<= 1e-12); smaller R show the truncation error"}


def run_layer(args, pj, world, rank, dev, stream, flush):
    """Config 5: forward and backward of the projected layer against cuBLAS BF16,
    every pass captured in a CUDA graph (the same for both sides)."""
    import synth
    X, W, dY = synth.layer_workload(seed=1)
    Xb = torch.from_numpy(X).to(dev).to(torch.bfloat16)
    Wb = torch.from_numpy(W).to(dev).to(torch.bfloat16)
    gb = torch.from_numpy(dY).to(dev).to(torch.bfloat16)
    M, K = Xb.shape
    N = Wb.shape[1]
    Kb, R = 256, 64
    Y = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    wsf = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R), dtype=torch.uint8, device=dev)
    wsb = torch.empty(pj.gemm_backward_workspace_size(M, N, K, Kb, R), dtype=torch.uint8, device=dev)
    Yc = torch.empty_like(Y)
    dXc = torch.empty_like(Xb)
    dWc = torch.empty_like(Wb)

    def fwd():
        pj.proj_gemm(Xb, Wb, Kb, R, out=Y, workspace=wsf, stream=torch.cuda.current_stream())

    def bwd():
        pj.proj_gemm_backward(Xb, Wb, gb, Kb, R, workspace=wsb, stream=torch.cuda.current_stream())

    def bwd_saved():   # from the projections the forward left in wsf
        pj.proj_gemm_backward_saved(wsf, gb, K, Kb, R, workspace=wsb, stream=torch.cuda.current_stream())

    def cub_fwd():
        torch.matmul(Xb, Wb, out=Yc)

    def cub_bwd():
        torch.matmul(gb, Wb.t(), out=dXc)
        torch.matmul(Xb.t(), gb, out=dWc)

    times = {}
    for name, fn in (("fwd", fwd), ("bwd", bwd), ("bwd_saved", bwd_saved), ("cub_fwd", cub_fwd),
                     ("cub_bwd", cub_bwd)):
        fn()
        g = _Direct(fn) if args.no_graph else capture(fn, stream)
        for _ in range(args.warmup):
            g.replay()
        (t,), _ = time_graphs([g], max(10, min(args.steps, 200)), flush, stream)
        times[name] = statistics.median(t)
    eff = 2.0 * M * N * K
    return {"workload": "layer X 8192x4096 @ W 4096x4096 bf16, block 256, R=64 (forward + backward)",
            "forward_ms": round(times["fwd"], 4), "backward_ms": round(times["bwd"], 4),
            "forward_eff_tflops": round(eff / (times["fwd"] * 1e-3) / 1e12, 1),
            "fwd_bwd_eff_tflops": round(3 * eff / ((times["fwd"] + times["bwd"]) * 1e-3) / 1e12, 1),
            "backward_saved_ms": round(times["bwd_saved"], 4),
            "fwd_bwd_saved_eff_tflops": round(3 * eff / ((times["fwd"] + times["bwd_saved"]) * 1e-3) / 1e12, 1),
            "cublas_bf16_forward_ms": round(times["cub_fwd"], 4), "cublas_bf16_backward_ms": round(times["cub_bwd"], 4),
            "timing": "direct calls" if args.no_graph else "CUDA graph replay per pass (ours and cuBLAS), L2 flushed"}


def run_batch(args, pj, world, rank, dev, stream, flush):
    """512 uneven GEMMs + 256 single-template correlations as one batched plan."""
    import synth
    gsz, csz = synth.uneven_batch_sizes(seed=0)
    if args.batch_fraction < 1.0:   # a smaller slice of the same batch (profiling captures)
        gsz = gsz[:max(1, int(len(gsz) * args.batch_fraction))]
        csz = csz[:max(1, int(len(csz) * args.batch_fraction))]
    Tc = 1024
    gem, cnv = [], []
    for i, (M, N, K) in enumerate(gsz):
        A = synth.device_normal((M, K), 2 * i + 1, dev)
        B = synth.device_normal((K, N), 2 * i + 2, dev)
        gem.append((A, B, torch.empty((M, N), device=dev)))
    for i, Sc in enumerate(csz):
        s = synth.device_normal((Sc,), 10000 + 2 * i, dev)
        k = synth.device_normal((1, Tc), 10001 + 2 * i, dev)
        cnv.append((s, k, torch.empty((Sc - Tc + 1, 1), device=dev)))
    eff = sum(2.0 * M * N * K for M, N, K in gsz) + sum(2.0 * (Sc - Tc + 1) * Tc for Sc in csz)
    rows = []

    def make_descs(Rg, Rc, split, compute):
        descs = [pj.batch_gemm(A, B, Y, 128, Rg, split=split, compute=compute) for A, B, Y in gem]
        return descs + [pj.batch_conv(s, k, o, Rc, split=split) for s, k, o in cnv]

    tuned = None
    if not args.no_tune:
        # the measuring autotuner: candidate tunings of the split BF16 plan, timed on the GPU
        best, trials = pj.autotune_batch(make_descs(128, 1024, 2, "bf16"), device=dev, stream=stream, reps=3)
        tuned = {"best": best, "trials": trials}
    settings = (("full R, split", 128, 1024, 2, "bf16", None),
                ("full R, split (untuned: 256-row tiles, round-robin)", 128, 1024, 2, "bf16",
                 {"schedule": 1, "tile_rows": 256}),
                ("full R", 128, 1024, 1, "bf16", None), ("R = block/2", 64, 512, 1, "bf16", None),
                ("full R, split, E4M3 GEMMs", 128, 1024, 2, "e4m3", None), ("full R, E4M3 GEMMs", 128, 1024, 1,
                                                                            "e4m3", None))
    for label, Rg, Rc, split, compute, tuning in settings:
        if args.batch_setting and args.batch_setting != label:
            continue
        if tuned is not None and tuning is None and compute == "bf16" and split == 2:
            tuning = tuned["best"]
        plan = pj.BatchPlan(make_descs(Rg, Rc, split, compute), device=dev, stream=stream, tuning=tuning)
        plan.run(stream)
        g = capture(lambda: plan.run(torch.cuda.current_stream()), stream)
        for _ in range(args.warmup):
            g.replay()
        (tms,), tot = time_graphs([g], args.steps, flush, stream)
        plan.check(stream)
        ms = tot / args.steps
        errs = []
        for A, B, Y in gem[:6]:
            errs.append(sampled_rel_err_gemm(A, B, Y))
        for s, k, o in cnv[:6]:
            errs.append(sampled_rel_err(s, k, o))
        rows.append({"setting": label, "R_gemm": Rg, "R_conv": Rc, "split": split, "gemm_compute": compute,
                     "tuning": tuning, "ms": round(ms, 3), "value": round(eff / (ms * 1e-3) / 1e12, 2),
                     "max_rel_err_sampled": max(errs), "plan": plan.info()})
        del plan, g
        torch.cuda.empty_cache()
    # A batch whose few tiles have a long reduced dimension: the tuner's K splits
    # spread them over the SMs (partial products added into the zeroed output).
    longk = []
    for i in range(0 if args.batch_setting else 2):
        A = synth.device_normal((512, 131072), 90001 + 2 * i, dev)
        B = synth.device_normal((131072, 512), 90002 + 2 * i, dev)
        longk.append((A, B, torch.empty((512, 512), device=dev)))
    eff_long = sum(2.0 * 512 * 512 * 131072 for _ in longk)
    long_rows = []
    for label, tuning in ((("tuned (K splits)", None), ("untuned", {"schedule": 1, "tile_rows": 256}))
                          if longk else ()):
        plan = pj.BatchPlan([pj.batch_gemm(A, B, Y, 128, 128) for A, B, Y in longk], device=dev, stream=stream,
                            tuning=tuning)
        plan.run(stream)
        g = capture(lambda: plan.run(torch.cuda.current_stream()), stream)
        for _ in range(args.warmup):
            g.replay()
        (tms,), tot = time_graphs([g], args.steps, flush, stream)
        plan.check(stream)
        ms = tot / args.steps
        long_rows.append({"setting": label, "ms": round(ms, 3), "value": round(eff_long / (ms * 1e-3) / 1e12, 2),
                          "rel_err_sampled": sampled_rel_err_gemm(*longk[0]), "plan": plan.info()})
        del plan, g
    del longk
    torch.cuda.empty_cache()
    base = []
    if not args.no_exact:
        import torch.nn.functional as F
        for name, tf32 in (("cublas tf32 + cudnn conv1d tf32", True), ("cublas fp32 + cudnn conv1d fp32", False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            torch.backends.cudnn.allow_tf32 = tf32

            def exact():
                for A, B, Y in gem:
                    torch.matmul(A, B, out=Y)
                for s, k, o in cnv:
                    F.conv1d(s.view(1, 1, -1), k.view(1, 1, -1))
            exact()
            torch.cuda.synchronize()
            ms = median_ms(exact, stream, flush, reps=3)
            errs = [sampled_rel_err_gemm(A, B, Y) for A, B, Y in gem[:6]]
            base.append({"impl": name, "ms": round(ms, 3), "value": round(eff / (ms * 1e-3) / 1e12, 2),
                         "max_rel_err_sampled_gemm": max(errs)})
        torch.backends.cuda.matmul.allow_tf32 = False
        torch.backends.cudnn.allow_tf32 = False
    return {"workload": "uneven batch: 512 GEMMs (M,N ~ U[64,2048], K ~ U[256,8192], block 128, DCT-II L=8) + "
                        "256 correlations (S ~ U[2^14,2^20], one template of 1024, Haar L=64), FP32 N(0,1) inputs",
            "effective_tflop_per_step": round(eff / 1e12, 3), "rows": rows, "autotune": tuned,
            "long_k": {"workload": "2 GEMMs 512x131072 by 131072x512, block 128, R = 128 (BF16)", "rows": long_rows},
            "exact_baselines": base,
            "timing": "CUDA graph of one proj_batch_run; inputs ~40 GB, far larger than L2"}


# ------------------------------------------ every config's <= 1e-3 headline --
# The default line carries, besides the CONV headline, one entry per other
# configuration of the method: its fastest setting whose sampled error against
# the exact FP64 result is at most 1e-3 (config 5 at its stated R), the exact
# cuBLAS / cuDNN comparators timed in the same run, and the step roofline
# t_roof / t with t_roof = max(F_alg / P, B_alg / HBM): F_alg = the reduced MMA
# flops of every pass plus the projection flops, B_alg = inputs read once plus
# outputs written once (projected intermediates not counted).

ARCH_BF16_FLOPS_PER_SM_CLK = 8192     # dense BF16 tensor-core rate of one SM per clock (sm_100 family)
SMS = 152


def step_roofline(F_alg, B_alg, ms, peak_tflops, hbm_gbs, peak_name):
    t_f = F_alg / (peak_tflops * 1e12) * 1e3
    t_b = B_alg / (hbm_gbs * 1e9) * 1e3
    t_roof = max(t_f, t_b)
    return {"bound": "tensor" if t_f >= t_b else "hbm", "t_roof_ms": round(t_roof, 4), "t_ms": round(ms, 4),
            "frac": round(t_roof / ms, 4), "F_alg_gflop": round(F_alg / 1e9, 2), "B_alg_mb": round(B_alg / 1e6, 1),
            "peak": f"{peak_name} {peak_tflops} TFLOP/s, HBM {hbm_gbs} GB/s (MEASURED_PEAKS.json)"}


def per_clock(flops, ms, sm_mhz):
    """Tensor-core flops per SM per clock at the sampled SM clock, against the architectural rate."""
    if not sm_mhz:
        return None
    r = flops / (ms * 1e-3) / (SMS * sm_mhz * 1e6)
    return {"flops_per_sm_clk": round(r, 1), "arch": ARCH_BF16_FLOPS_PER_SM_CLK,
            "frac": round(r / ARCH_BF16_FLOPS_PER_SM_CLK, 4), "sm_mhz": sm_mhz}


def best_exact(base):
    ok = [b for b in base if "ms" in b and b.get("rel_err_vs_exact", 1.0) <= 1e-3]
    return min(ok, key=lambda b: b["ms"]) if ok else None


def config_face(pj, dev, stream, flush, steps, warmup):
    """Config 3: 4096 x 10304 face probes by a 10304 x 2048 orthonormal feature matrix, block 512."""
    import synth
    hbm, _, bf16_sus, _ = peaks()
    M, K, N, Kb = 4096, 10304, 2048, 512
    A = torch.from_numpy(synth.face_probes(M, seed=0)).to(dev)
    B = torch.from_numpy(synth.orthonormal_features(K, N, seed=1)).to(dev)
    eff = 2.0 * M * N * K
    rows = []

    def reduced_k(R, split, lead):
        kp = R * (K // Kb) + (R // (Kb // 8)) * ((K % Kb) // 8)
        kt = kp // (R // (Kb // 8)) * lead if lead else kp
        return kp + (2 * kt if split == 2 else 0)

    # (R, split, lead, feature matrix cached, FP8 tier of truncated projections, A projected inside the GEMM)
    for R, split, lead, cached, tier, fused in ((512, 2, 1, False, 0, False), (512, 2, 1, True, 0, False),
                                                (512, 2, 0, False, 0, False), (512, 2, 0, True, 0, False),
                                                (512, 2, 0, True, 0, True), (512, 1, 0, True, 0, False),
                                                (512, 1, 0, True, 0, True),
                                                (128, 1, 0, False, 0, False), (64, 1, 0, False, 0, False),
                                                (128, 1, 0, False, 6, False), (128, 2, 1, False, 6, False),
                                                (64, 1, 0, False, 7, False)):
        ws = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R, split=split, split_lead=lead, fp8_tier=tier),
                         dtype=torch.uint8, device=dev)
        Y = torch.empty((M, N), dtype=torch.float32, device=dev)
        if cached:   # the feature matrix projected once, outside the timed steps
            pj.proj_gemm_project(None, B, Kb, R, ws, split=split, M=M, N=N, K=K, split_lead=lead, fp8_tier=tier)

        def gp():
            if not fused:
                pj.proj_gemm_project(A, None if cached else B, Kb, R, ws, split=split, N=N, split_lead=lead,
                                     stream=torch.cuda.current_stream(), fp8_tier=tier)

        def gm():
            if fused:
                pj.proj_gemm_fused(A, Y, Kb, R, ws, split=split, stream=torch.cuda.current_stream())
            else:
                pj.proj_gemm_multiply(Y, K, Kb, R, ws, split=split, split_lead=lead,
                                      stream=torch.cuda.current_stream(), fp8_tier=tier)

        gp()
        gm()
        gs = [capture(gm, stream)] if fused else [capture(gp, stream), capture(gm, stream)]
        for _ in range(warmup):
            for g in gs:
                g.replay()
        parts, tot = time_graphs(gs, steps, flush, stream)
        pm, mm = ([0.0], parts[0]) if fused else parts
        pj.check(ws)
        ms = tot / steps
        red = 2.0 * M * N * reduced_k(R, split, lead)
        lp1 = R // (Kb // 8)
        # the FP8 tier's products count at half weight: the E4M3 tensor rate is twice the BF16 one
        red8 = 2.0 * M * N * reduced_k(tier * (Kb // 8), 1, 0) if tier else 0.0
        F = red + red8 / 2 + 2.0 * (M + (0 if cached else N)) * K * (lp1 + tier)
        # cached: the projected feature matrix B_d (N rows of the reduced pitch, BF16) is read instead of B
        Bytes = 4.0 * (M * K + M * N) + (2.0 * N * reduced_k(R, split, lead) if cached else 4.0 * K * N)
        mmed = statistics.median(mm)
        rows.append({"R": R, "split": split, "split_lead": lead, "fp8_tier": tier,
                     "setting": ("feature matrix projected once (per probe batch)" if cached else "one call")
                     + (", probes projected inside the GEMM (fused)" if fused else "")
                     + (f", projections {lp1}..{lp1 + tier - 1} added in E4M3" if tier else ""),
                     "ms": round(ms, 4), "value": round(eff / (ms * 1e-3) / 1e12, 2),
                     "project_ms": round(statistics.median(pm), 4), "multiply_ms": round(mmed, 4),
                     "rel_err_vs_exact": sampled_rel_err_gemm(A, B, Y),
                     "roofline": step_roofline(F, Bytes, ms, bf16_sus, hbm, "bf16 sustained"),
                     "gemm_kernel": {"kernel": ("gemm_fused_kernel" if fused else "gemm_cg2_kernel")
                                     + (" + gemm_mx_kernel" if tier else ""),
                                     "ms": round(mmed, 4),
                                     "tflops_reduced": round((red + red8) / (mmed * 1e-3) / 1e12, 1),
                                     "flops": red + red8 / 2}})
        del ws, Y, gs
    base = gemm_exact_baselines(A, B, stream, flush)
    return headline_entry("face-gemm 4096x10304 by 10304x2048, block 512, DCT-II L=8 (BF16 components)", rows, base)


def headline_entry(workload, rows, base):
    ok = [r for r in rows if r.get("rel_err_vs_exact", 1.0) <= 1e-3]
    best = min(ok, key=lambda r: r["ms"]) if ok else None
    ex = best_exact(base)
    out = {"workload": workload, "headline": best, "fastest_exact_at_1e-3": ex,
           "speedup_vs_exact": round(ex["ms"] / best["ms"], 3) if best and ex else None,
           "rows": rows, "exact_baselines": base}
    return out


def config_layer(pj, dev, stream, flush, steps, warmup):
    """Config 5: forward and backward of X 8192x4096 @ W 4096x4096 (BF16), block 256, R = 64."""
    import synth
    hbm, _, bf16_sus, _ = peaks()
    X, W, dY = synth.layer_workload(seed=1)
    Xb = torch.from_numpy(X).to(dev).to(torch.bfloat16)
    Wb = torch.from_numpy(W).to(dev).to(torch.bfloat16)
    gb = torch.from_numpy(dY).to(dev).to(torch.bfloat16)
    M, K = Xb.shape
    N = Wb.shape[1]
    Kb, R = 256, 64
    Kp = K * R // Kb
    Y = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    dX = torch.empty_like(Xb)
    dW = torch.empty_like(Wb)
    wsf = torch.empty(pj.gemm_workspace_size(M, N, K, Kb, R), dtype=torch.uint8, device=dev)
    wsb = torch.empty(pj.gemm_backward_workspace_size(M, N, K, Kb, R), dtype=torch.uint8, device=dev)
    Yc, dXc, dWc = torch.empty_like(Y), torch.empty_like(Xb), torch.empty_like(Wb)
    fns = {"fwd": lambda: pj.proj_gemm(Xb, Wb, Kb, R, out=Y, workspace=wsf, stream=torch.cuda.current_stream()),
           "bwd": lambda: pj.proj_gemm_backward(Xb, Wb, gb, Kb, R, workspace=wsb, stream=torch.cuda.current_stream(),
                                                dA=dX, dB=dW),
           # the forward's workspace still holds X_c and W_d: the training-step form
           "bwd_saved": lambda: pj.proj_gemm_backward_saved(wsf, gb, K, Kb, R, workspace=wsb,
                                                            stream=torch.cuda.current_stream(), dA=dX, dB=dW),
           "cub_fwd": lambda: torch.matmul(Xb, Wb, out=Yc),
           "cub_bwd": lambda: (torch.matmul(gb, Wb.t(), out=dXc), torch.matmul(Xb.t(), gb, out=dWc))}
    t = {}
    for name, fn in fns.items():
        fn()
        g = capture(fn, stream)
        for _ in range(warmup):
            g.replay()
        (tt,), _ = time_graphs([g], max(10, steps), flush, stream)
        t[name] = statistics.median(tt)
    eff = 2.0 * M * N * K
    red = 2.0 * M * N * Kp
    lp1 = R // (Kb // 8)
    MiB = 2.0 ** 20
    F_f = red + 2.0 * (M + N) * K * lp1
    F_b = 2 * red + 2.0 * (M + N) * K * lp1 * 2
    rel = sampled_rel_err_gemm(Xb.float(), Wb.float(), Y.float())
    return {"workload": "layer X 8192x4096 @ W 4096x4096 bf16, block 256, R=64 (forward + backward)",
            "note": "judged on gradient correctness (tests) and throughput; the truncation error at R/block = 1/4 "
                    "of Gaussian data is about sqrt(3/4), so 1e-3 does not apply",
            "forward": {"ms": round(t["fwd"], 4), "value": round(eff / (t["fwd"] * 1e-3) / 1e12, 1),
                        "rel_err_vs_exact": rel,
                        "roofline": step_roofline(F_f, (64 + 32 + 64) * MiB, t["fwd"], bf16_sus, hbm,
                                                  "bf16 sustained")},
            "backward": {"ms": round(t["bwd"], 4), "value": round(2 * eff / (t["bwd"] * 1e-3) / 1e12, 1),
                         "roofline": step_roofline(F_b, (64 + 32 + 64 + 64 + 32) * MiB, t["bwd"], bf16_sus, hbm,
                                                   "bf16 sustained")},
            # backward from the forward's saved projections (proj_gemm_backward_saved): the
            # two reduced products and their expansion only; X and W are not read again
            "backward_saved": {"ms": round(t["bwd_saved"], 4),
                               "value": round(2 * eff / (t["bwd_saved"] * 1e-3) / 1e12, 1),
                               "roofline": step_roofline(2 * red, (16 + 8 + 64 + 64 + 32) * MiB, t["bwd_saved"],
                                                         bf16_sus, hbm, "bf16 sustained")},
            "cublas_bf16": {"forward_ms": round(t["cub_fwd"], 4), "backward_ms": round(t["cub_bwd"], 4)},
            "speedup_vs_cublas_bf16": {"forward": round(t["cub_fwd"] / t["fwd"], 3),
                                       "backward": round(t["cub_bwd"] / t["bwd"], 3),
                                       "backward_saved": round(t["cub_bwd"] / t["bwd_saved"], 3),
                                       "forward_plus_backward": round((t["cub_fwd"] + t["cub_bwd"])
                                                                      / (t["fwd"] + t["bwd"]), 3),
                                       "forward_plus_backward_saved": round((t["cub_fwd"] + t["cub_bwd"])
                                                                            / (t["fwd"] + t["bwd_saved"]), 3)},
            "forward_flops": red}


def config_fp64(pj, dev, stream, flush, steps, warmup):
    """Config 1: FP64 projected GEMM, A 256x512 by B 512x256 (uniform [-1, 1)), block 128, DCT-II L = 8."""
    import synth
    hbm = peaks()[0]
    A_np, B_np = synth.uniform_pair(256, 512, 256, seed=0)
    A = torch.from_numpy(A_np).to(dev)
    B = torch.from_numpy(B_np).to(dev)
    exact = A @ B
    # the FP64 rate of this GPU, measured here on a large cuBLAS DGEMM (the roofline's P)
    big = torch.randn((4096, 4096), dtype=torch.float64, device=dev)
    dg = median_ms(lambda: torch.matmul(big, big), stream, flush, reps=3)
    p64 = 2.0 * 4096 ** 3 / (dg * 1e-3) / 1e12
    del big
    rows = []
    for R in (128, 64, 32, 16):
        Y = torch.empty((256, 256), dtype=torch.float64, device=dev)
        ws = torch.empty(pj.gemm_workspace_size(256, 256, 512, 128, R, compute="f64"), dtype=torch.uint8, device=dev)

        def fn():
            pj.proj_gemm(A, B, 128, R, compute="f64", out=Y, workspace=ws, stream=torch.cuda.current_stream())

        fn()
        g = capture(fn, stream)
        for _ in range(warmup):
            g.replay()
        (tt,), _ = time_graphs([g], max(10, steps), flush, stream)
        ms = statistics.median(tt)
        F = 2.0 * 256 * 256 * 512 * R / 128 + 2.0 * (256 + 256) * 512 * (R // 16)
        rows.append({"R": R, "ms": round(ms, 4), "value": round(2.0 * 256 * 256 * 512 / (ms * 1e-3) / 1e12, 4),
                     "rel_err_vs_exact": float(torch.linalg.norm(Y - exact) / torch.linalg.norm(exact)),
                     "roofline": step_roofline(F, 8.0 * (2 * 256 * 512 + 256 * 256), ms, round(p64, 2), hbm,
                                               "fp64 (cuBLAS DGEMM 4096^3 measured in this run)")})
    Yx = torch.empty_like(exact)
    ms = median_ms(lambda: torch.matmul(A, B, out=Yx), stream, flush, reps=5)
    base = [{"impl": "cublas fp64", "ms": round(ms, 4), "value": round(2.0 * 256 * 256 * 512 / (ms * 1e-3) / 1e12, 4),
             "rel_err_vs_exact": 0.0}]
    out = headline_entry("fp64 GEMM 256x512 by 512x256, uniform[-1,1), block 128, DCT-II L=8", rows, base)
    out["note"] = ("a correctness configuration (latency-bound at this size): full R must equal the FP64 product "
                   "to 1e-12; smaller R show the truncation error of i.i.d. data")
    return out


def config_batch(pj, dev, stream, flush, steps, warmup):
    """Config 4: 512 uneven GEMMs + 256 single-template correlations in one plan (CUDA graph)."""
    import synth
    import torch.nn.functional as F
    hbm, _, bf16_sus, _ = peaks()
    gsz, csz = synth.uneven_batch_sizes(seed=0)
    Tc = 1024
    gem, cnv = [], []
    for i, (M, N, K) in enumerate(gsz):
        gem.append((synth.device_normal((M, K), 2 * i + 1, dev), synth.device_normal((K, N), 2 * i + 2, dev),
                    torch.empty((M, N), device=dev)))
    for i, Sc in enumerate(csz):
        cnv.append((synth.device_normal((Sc,), 10000 + 2 * i, dev), synth.device_normal((1, Tc), 10001 + 2 * i, dev),
                    torch.empty((Sc - Tc + 1, 1), device=dev)))
    eff = sum(2.0 * M * N * K for M, N, K in gsz) + sum(2.0 * (Sc - Tc + 1) * Tc for Sc in csz)
    B_alg = sum(4.0 * (M * K + K * N + M * N) for M, N, K in gsz) + sum(4.0 * (2 * Sc - Tc + 1 + Tc) for Sc in csz)
    rows = []
    for label, Rg, Rc, split in (("full R, split (BF16)", 128, 1024, 2), ("full R (BF16)", 128, 1024, 1)):
        descs = [pj.batch_gemm(A, B, Y, 128, Rg, split=split) for A, B, Y in gem]
        descs += [pj.batch_conv(s_, k_, o_, Rc, split=split) for s_, k_, o_ in cnv]
        plan = pj.BatchPlan(descs, device=dev, stream=stream)
        plan.run(stream)
        g = capture(lambda: plan.run(torch.cuda.current_stream()), stream)
        for _ in range(warmup):
            g.replay()
        (tms,), tot = time_graphs([g], steps, flush, stream)
        plan.check(stream)
        ms = tot / steps
        errs = [sampled_rel_err_gemm(A, B, Y) for A, B, Y in gem[:8]] + [sampled_rel_err(s_, k_, o_)
                                                                           for s_, k_, o_ in cnv[:8]]
        npass = 3 if split == 2 else 1
        F_alg = npass * eff + sum(2.0 * (M + N) * K * 8 for M, N, K in gsz)
        rows.append({"setting": label, "ms": round(ms, 3), "value": round(eff / (ms * 1e-3) / 1e12, 2),
                     "rel_err_vs_exact": max(errs), "error_is": "largest sampled relative error of 16 instances",
                     "roofline": step_roofline(F_alg, B_alg, ms, bf16_sus, hbm, "bf16 sustained"),
                     "plan": plan.info()})
        del plan, g
        torch.cuda.empty_cache()
    base = []
    for name, tf32 in (("cublas tf32 + cudnn conv1d tf32", True), ("cublas fp32 + cudnn conv1d fp32", False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        torch.backends.cudnn.allow_tf32 = tf32

        def exact():
            for A, B, Y in gem:
                torch.matmul(A, B, out=Y)
            for s_, k_, o_ in cnv:
                o_.copy_(F.conv1d(s_.view(1, 1, -1), k_.view(1, 1, -1)).view(-1, 1))
        exact()
        torch.cuda.synchronize()
        ms = median_ms(exact, stream, flush, reps=3)
        errs = [sampled_rel_err_gemm(A, B, Y) for A, B, Y in gem[:8]] + [sampled_rel_err(s_, k_, o_)
                                                                           for s_, k_, o_ in cnv[:8]]
        base.append({"impl": name, "ms": round(ms, 3), "value": round(eff / (ms * 1e-3) / 1e12, 2),
                     "rel_err_vs_exact": max(errs)})
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.backends.cudnn.allow_tf32 = False
    del gem, cnv
    torch.cuda.empty_cache()
    return headline_entry("uneven batch: 512 GEMMs (M,N ~ U[64,2048], K ~ U[256,8192], block 128, DCT-II L=8) + "
                          "256 correlations (S ~ U[2^14,2^20], one template of 1024, Haar L=64), FP32 N(0,1) inputs, "
                          "one plan per step (CUDA graph), inputs ~40 GB", rows, base)


def run_configs(args, pj, dev, stream, flush):
    """Every other configuration's <= 1e-3 headline, exact comparators and roofline (rank 0, after the timed
    CONV steps)."""
    clocks = ClockSampler(dev.index)
    clocks.start()
    steps, warmup = max(10, min(args.steps, 50)), args.warmup
    out = {}
    out["config3_face_gemm"] = config_face(pj, dev, stream, flush, steps, warmup)
    out["config5_layer"] = config_layer(pj, dev, stream, flush, steps, warmup)
    out["config1_fp64"] = config_fp64(pj, dev, stream, flush, steps, warmup)
    if not args.no_batch_config:
        out["config4_batch"] = config_batch(pj, dev, stream, flush, max(5, min(args.steps, 10)), warmup)
    out["clocks"] = clk = clocks.stop()
    # tensor-core rate per SM and clock at this section's median sampled SM clock
    for r in out["config3_face_gemm"]["rows"]:
        k = r["gemm_kernel"]
        k["per_clock"] = per_clock(k.pop("flops"), k["ms"], clk.get("sm_mhz"))
    lay = out["config5_layer"]
    lay["forward"]["per_clock"] = per_clock(lay.pop("forward_flops"), lay["forward"]["ms"], clk.get("sm_mhz"))
    return out


def library_variant(world: int) -> str:
    """The library build a rank loads: with one process per GPU on several GPUs,
    the build without CTA pairs, which holds no cluster-multicast form."""
    return "solo" if world > 1 else "pairs"


def run_ours(args):
    import paper_1411_2860_gb300 as pj
    world, rank, local = dist_env()
    pj.select_library(library_variant(world))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pj.build()
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    torch.backends.cuda.matmul.allow_tf32 = False
    with torch.cuda.stream(stream):
        if args.workload == "conv":
            line = run_conv(args, pj, world, rank, dev, stream, flush)
        else:
            fn = {"face-gemm": run_face_gemm, "layer": run_layer, "batch": run_batch,
                  "fp64": run_fp64}[args.workload]
            line = fn(args, pj, world, rank, dev, stream, flush) if rank == 0 else None
    if line is not None and args.workload == "conv" and not args.no_configs:
        args._sm_mhz = line["clocks"].get("sm_mhz")
        line["roofline"]["per_clock"] = per_clock(2.0 * LAGS * NT * args.R, line["roofline"]["kernel_ms"],
                                                  args._sm_mhz)
        with torch.cuda.stream(stream):
            line["configs"] = run_configs(args, pj, dev, stream, flush)
    if line is not None and args.workload == "conv" and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if world > 1:
        torch.distributed.destroy_process_group()
    return line


def _oracle_sample(seconds):
    import oracle
    import synth
    s, k, _ = synth.audio_workload(S, T, NT, seed=0)
    s64, k64 = s.astype(np.float64), k.astype(np.float64)
    n = 2048
    t0 = time.perf_counter()
    oracle.conv_proj(s64[:n + T - 1], k64, 4096, "haar", L)
    dt = time.perf_counter() - t0
    n = int(max(256, min(LAGS, n * seconds / max(dt, 1e-3))))
    return oracle, s64, k64, n


def cpu_baseline(seconds=10.0, R=4096):
    """FP64 oracle, as it stands, on a contiguous run of lags of the same workload."""
    oracle, s64, k64, n = _oracle_sample(seconds)
    t0 = time.perf_counter()
    oracle.conv_proj(s64[:n + T - 1], k64, R, "haar", L)
    dt = time.perf_counter() - t0
    return {"value": round(2.0 * n * NT * T / dt / 1e12, 6), "unit": "TFLOP/s", "cores": oracle.threads(),
            "kind": "oracle", "sample": f"{n} consecutive lags x {NT} templates at R={R} (FP64, all cores)",
            "seconds": round(dt, 2)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    per_step = min(10.0, max(1.0, 60.0 / max(1, args.steps + args.warmup)))
    oracle, s64, k64, n = _oracle_sample(per_step)
    R = args.R or 4096
    for _ in range(args.warmup):
        oracle.conv_proj(s64[:n + T - 1], k64, R, "haar", L)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.conv_proj(s64[:n + T - 1], k64, R, "haar", L)
    dt = time.perf_counter() - t0
    value = 2.0 * n * NT * T * args.steps / dt / 1e12
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"projected cross-correlation: audio-like signal 2^20 samples x 64 templates "
                               f"of 4096, Haar L=64, R={R}, sample of {n} lags per step",
                   "S": S, "T": T, "n_templates": NT, "R": R},
        "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "kind": "oracle", "cores": oracle.threads(),
                         "sample": f"{n} consecutive lags x {NT} templates per step"},
        "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["conv", "face-gemm", "layer", "batch", "fp64"], default="conv")
    ap.add_argument("--R", type=int, default=None)
    ap.add_argument("--split", type=int, default=1)
    ap.add_argument("--compute", choices=["bf16", "e4m3"], default=None)
    ap.add_argument("--split-lead", type=int, default=0, help="face-gemm: lo term on projections p < this only")
    ap.add_argument("--fused", action="store_true", help="face-gemm: B projected once, A projected inside the GEMM "
                                                         "(proj_gemm_fused; R = block)")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: skip the measuring autotuner")
    ap.add_argument("--batch-fraction", type=float, default=1.0,
                    help="batch workload: run only this fraction of the instances (profiling)")
    ap.add_argument("--batch-setting", default=None, help="batch workload: run only the settings whose label "
                                                          "contains this text")
    ap.add_argument("--conv-basis", choices=["haar", "dct2"], default="haar",
                    help="conv workload: projection basis (Haar: the box path; DCT-II: the general path)")
    ap.add_argument("--conv-L", type=int, default=64, help="conv workload: group size L of the basis")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="conv workload: leave out the other configurations")
    ap.add_argument("--no-batch-config", action="store_true", help="leave out config 4 (about 40 GB of inputs)")
    ap.add_argument("--no-exact", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload == "conv" and args.R is None:
        args.R = 4096
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
