"""The multi-rank benchmark path on CPU (gloo, world size 2): every rank
dedisperses its own beam of the same shape (weak scaling, no data-path
collective); the job's time is the largest rank time and its throughput the
units all ranks processed over it; only rank 0 prints.  The GPU work itself
needs a GB300 and is covered by the -m gpu tests."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own beam: same shape, different data
        w = synth.WORKLOADS["fdd_64ch_4096t_128dm"].scaled(fixed_pulse=None)
        fb, _ = synth.filterbank(w, seed=20211007, beam=rank, rows=256)
        ms = 10.0 + 5.0 * rank  # rank times of a step
        ms_max = bench.max_over_ranks(dist, ms, "cpu")
        rate = bench.job_rate(1.0e9, 4, world, ms_max)
        q.put((rank, float(fb.astype(np.float64).sum()), ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, v0), (r1, s1, m1, v1) = out
    assert (r0, r1) == (0, 1) and s0 != s1            # distinct beams per rank
    assert m0 == m1 == 15.0                           # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(1.0e9 * 4 * 2 / 0.015)


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node",
           "2", "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "fdd_64ch_4096t_128dm"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
