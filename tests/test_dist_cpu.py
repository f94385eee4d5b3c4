"""The multi-rank path of bench.py on the host: world_size-2 process groups
over gloo on 127.0.0.1.  The path shards by waveform (independent problems,
no data-path collective), so what runs across ranks is the timing reduction
(max over ranks), the disjoint waveform sets, the whole-job rate, and the
reference arm's rank-0-only output under torchrun."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    seeds = bench.rank_seeds(rank, 8)
    allseeds = [None] * world
    dist.all_gather_object(allseeds, seeds)
    rate = bench.job_rate(60, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, allseeds, rate))


def test_gloo_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, allseeds, rate in res:
        assert ms == 15.0                                   # the slowest rank's time, on every rank
        assert set(allseeds[0]).isdisjoint(allseeds[1])     # independent waveforms per rank
        assert len(allseeds[0]) == len(allseeds[1]) == 8    # the same work per rank (weak scaling)
        assert rate == pytest.approx(2 * 60 / 0.015)        # units of all ranks over the max time


def test_reference_arm_under_torchrun():
    """`bench.py --impl reference` launched as two ranks: rank 0 alone prints one
    JSON line (the CPU oracle timed on the host), the other rank exits 0."""
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
