"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The method shards as independent disorder samples (replicas only, no data
collective): each rank gets its own seed, the timed region's slowest rank
sets the time, and the whole-job rate counts every rank's updates.  The
reference arm runs on rank 0 alone; the other ranks exit without work."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank], dist, "cpu")
    out[rank] = (got, bench.rank_seed(3, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_rank_seeds_with_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == [2.0, 10.0, 0.5]
    assert res[0][1] != res[1][1]


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1e6, 4, 2.0) == pytest.approx(4e6 / 2e6)
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]


def test_reference_arm_under_two_ranks_prints_one_line():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "L6_Lt32_single", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
