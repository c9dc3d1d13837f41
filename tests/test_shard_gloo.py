"""One text scanned by 2 and 3 gloo ranks on CPU (the paper's Section 4.3
split, Eq. 3, and its reduction of the counts): each rank scans its piece
with the library's host walk of the compiled tables, the counts are summed
and the rank-ordered keys gathered, and the merged result equals the
oracle's for the whole text -- including matches that straddle a split
point and pieces shorter than a pattern. No GPU is used."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1407_2889_gb300 import shard, synth  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(kind):
    T = synth.est_text(1 << 15, 21)
    if kind == "runs":
        # one letter across every split point: every window there matches
        T = np.full(6001, ord("A"), np.uint8)
        P = np.array([[ord("A")] * 7, list(b"AAAAAAC"), [ord("A")] * 7], np.uint8)
        return T, P, "ac"
    P = synth.mixed_patterns(T, 120, 9, 21)
    P = np.concatenate([P, P[:4]])  # duplicates
    if kind == "tiny":
        return T[:11], P, "ac"      # pieces shorter than a pattern
    return T, P, kind


def _worker(rank, world, port, kind, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1407_2889_gb300 import pmscan as pm
        T, P, algo = _case(kind)
        host = {"host_only": 1}
        s = pm.PatternSet.ac(P, host) if algo == "ac" else pm.PatternSet.wm(P, 3, host)
        occ, counts = shard.sharded_scan(s.h, T, P.shape[1], dist, host_walk=True)
        q.put((rank, occ.tobytes(), counts.tobytes()))
        s.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("kind", ["ac", "wm", "runs", "tiny"])
def test_sharded_scan_equals_the_whole_text(world, kind):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    T, P, _ = _case(kind)
    want_occ, want_cnt = oracle.dictionary(T, P, threads=2)
    for rank, occ_b, cnt_b in res:
        occ = np.frombuffer(occ_b, np.uint64)
        cnt = np.frombuffer(cnt_b, np.int64)
        assert np.array_equal(occ, want_occ), f"rank {rank}: merged occurrences"
        assert np.array_equal(cnt, want_cnt), f"rank {rank}: summed counts"


def test_pieces_cover_every_start_once():
    for n in (0, 1, 7, 8, 9, 100, 12345):
        for m in (1, 3, 8):
            for world in (1, 2, 3, 5):
                owned = []
                for r in range(world):
                    a, b, c = shard.piece(n, m, r, world)
                    assert a <= b <= c <= n and c - b <= m - 1
                    owned.extend(range(a, b))
                assert owned == list(range(n))
