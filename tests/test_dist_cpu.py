"""Multi-rank host logic of bench.py on CPU: two gloo ranks, no GPU.

Each rank runs an independent instance (weak scaling); the only cross-rank
operations are the barrier and the max-over-ranks timer.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    w, r, _ = bench.dist_env()
    ms = 10.0 + 5.0 * rank                       # rank 1 is slower
    slowest = bench.reduce_max(ms, w, torch.device("cpu"))
    value = bench.job_throughput(w, 7, slowest)
    s, _, _ = synth.audio_workload(4096, 256, 2, seed=r)   # each rank seeds its own instance
    dist.barrier()

    class A:
        steps, warmup, R = 1, 0, 4096
    ref = bench.run_reference(A)   # rank 0 times a bounded oracle sample; the other ranks return None
    q.put((r, w, slowest, value, float(s[:16].sum()), ref))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_timer_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, m0, v0, s0, ref0), (r1, w1, m1, v1, s1, ref1) = res
    assert (w0, w1) == (2, 2)
    assert m0 == m1 == 15.0                      # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 2.0 * (2**20 - 4095) * 64 * 4096 * 7 / 15e-3 / 1e12)
    assert s0 != s1                              # independent inputs per rank
    assert ref1 is None                          # the reference arm runs on rank 0 only
    # the reference arm's JSON line carries the contract's keys
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in ref0, key
    assert ref0["impl"] == "reference" and ref0["n_gpus"] == 2 and ref0["value"] > 0
    assert ref0["cpu_baseline"]["kind"] == "oracle" and ref0["cpu_baseline"]["cores"] >= 1
    assert ref0["e2e"]["h2d_bytes_per_step"] == 0 and ref0["e2e"]["value"] == ref0["value"]
