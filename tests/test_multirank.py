"""The bench's multi-rank host logic on CPU with two gloo ranks (the GPU runs
use one process per GPU over NCCL; replicas, no collective on the data path):
the max over ranks of a time, the whole-job throughput, distinct per-rank
seeds, and the reference arm running on rank 0 alone."""
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


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.rank_env()
    elapsed = [120.0, 150.0][rank]                       # rank 1 is the slow one
    mx = bench.max_over_ranks(elapsed, w, torch.device("cpu"))
    value = bench.whole_job_value(w, 64, 10, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, mx, value, bench.rank_seed(r)))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, mx, value, seed) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert mx == 150.0                                # every rank sees the slowest time
        assert value == pytest.approx(2 * 64 * 10 / 0.150)
    assert out[0][5] != out[1][5]                         # replicas draw different inputs


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_value(1, 64, 60, 1000.0) == pytest.approx(3840.0)
    assert bench.rank_seed(0) == 2


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""                         # only rank 0 prints the JSON line
    with pytest.raises(json.JSONDecodeError):
        json.loads(r.stdout or "x")
