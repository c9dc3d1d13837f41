"""The N>1 path of bench.py on CPU: two gloo ranks (replicas), barrier,
max-over-ranks timing and the whole-job rate, and the reference arm printing
on rank 0 only. No GPU is used."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        mine = [12.5, 40.0][rank]          # rank 1 is the slow one
        got = bench.max_over_ranks(mine, dist, torch, "cpu")
        rate = bench.job_rate(1 << 30, 10, world, got)
        q.put((rank, got, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, got, rate in res:
        assert got == 40.0
        assert rate == pytest.approx(2 * (1 << 30) * 10 / 0.040 / 1e9)


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun every rank but 0 exits 0 without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0"],
                         env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_job_rate_is_weak_scaling():
    one = bench.job_rate(1 << 30, 400, 1, 1000.0)
    two = bench.job_rate(1 << 30, 400, 2, 1000.0)
    assert two == pytest.approx(2 * one)
    assert json.dumps({"v": one})
