"""One text scanned by several ranks: the node split of the paper's Section
4.3 (Eq. 3) and its reduction of the counts, for ranks of torch.distributed.

Rank k of N owns the start positions [k n / N, (k+1) n / N) and reads its
range plus the m-1 bytes after it (the paper's stop = (rank+1) n / size +
(m-1)), clamped at n; every start position belongs to exactly one rank.
Each rank scans its piece with the library (on its own GPU, or with the
library's host walk of the compiled tables where no GPU is present), keeps
the occurrences that start in its own range, and shifts their positions by
its start. The per-pattern counts are then summed over the ranks (the
paper's MPI_Reduce, here an all-reduce) and the rank-ordered key lists are
gathered: each rank's keys are sorted and its positions lie below the next
rank's, so concatenation in rank order is the sorted list of the whole
text. The exchange carries d counts and the keys; tables are compiled on
every rank.
"""
from __future__ import annotations

import numpy as np

from . import pmscan as pm


def piece(n: int, m: int, rank: int, world: int) -> tuple[int, int, int]:
    """(start, own_end, read_end) of a rank: it owns start positions
    [start, own_end) and reads bytes [start, read_end)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    start = rank * n // world
    own_end = (rank + 1) * n // world
    read_end = min(n, own_end + m - 1)
    return start, own_end, read_end


def local_scan(handle: int, T: np.ndarray, m: int, rank: int, world: int, host_walk: bool = False):
    """This rank's part of the result: (keys with global positions, counts)
    of the occurrences that start in its own range."""
    start, own_end, read_end = piece(int(T.size), m, rank, world)
    part = np.ascontiguousarray(T[start:read_end])
    occ, counts = (pm.pm_selfcheck_host_walk(handle, part) if host_walk else pm.pm_scan(handle, part))
    occ = np.asarray(occ, dtype=np.uint64)
    pos = (occ >> np.uint64(32)).astype(np.int64)
    keep = pos < own_end - start
    if not keep.all():
        # an occurrence that starts in the overlap belongs to the next rank
        dropped = occ[~keep] & np.uint64(0xFFFFFFFF)
        counts = counts.copy()
        np.subtract.at(counts, dropped.astype(np.int64), 1)
        occ = occ[keep]
    occ = occ + (np.uint64(start) << np.uint64(32))
    return occ, np.asarray(counts, dtype=np.int64)


def merge(occ: np.ndarray, counts: np.ndarray, dist, group=None, device=None):
    """Sum the counts over the ranks and gather the rank-ordered keys on
    every rank (lengths first, then the keys padded to the longest).
    Returns (occ of the whole text, counts of the whole text)."""
    import torch

    world = dist.get_world_size(group)
    dev = device or "cpu"
    c = torch.from_numpy(np.ascontiguousarray(counts, dtype=np.int64)).to(dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    ln = torch.tensor([int(occ.size)], dtype=torch.int64, device=dev)
    lens = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(lens, ln, group=group)
    lens = [int(x.item()) for x in lens]
    longest = max(lens) if lens else 0
    mine = torch.zeros(max(longest, 1), dtype=torch.int64, device=dev)
    if occ.size:
        mine[: occ.size] = torch.from_numpy(occ.view(np.int64)).to(dev)
    parts = [torch.zeros(max(longest, 1), dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    keys = np.concatenate([p[:k].cpu().numpy() for p, k in zip(parts, lens)]).view(np.uint64)
    return keys, c.cpu().numpy()


def sharded_scan(handle: int, T: np.ndarray, m: int, dist, group=None, host_walk: bool = False, device=None):
    """The whole text's result, scanned by the ranks of `group` in Eq. 3
    pieces. Every rank passes the same text (or at least its own piece in
    place: only T[start:read_end] of this rank is read)."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    occ, counts = local_scan(handle, T, m, rank, world, host_walk=host_walk)
    return merge(occ, counts, dist, group=group, device=device)
