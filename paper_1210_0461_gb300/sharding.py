"""Sharding the product over several GPUs by partition interval.

Section 4 ("Our approach") and Theorem 1: K instances of CRoP, each with a
disjoint interval of the hash table and a full copy of the input, need no
communication while they accumulate; every entry is produced by exactly one
instance.  The heaviest entries of the whole product are then the heaviest of
the union of every instance's own heaviest entries, which is the only exchange
(a gather of k candidates per rank).  The per-partition Count-Sketch of an
interval plan holds estimators for its own partitions only (zero elsewhere),
so the whole sketch is the sum of the ranks' sketches.
"""
from __future__ import annotations

import numpy as np


def partition_interval(rank: int, world: int, P: int) -> tuple[int, int]:
    """Rank's equal share [q, r) of the P partitions (world <= P)."""
    if not 0 <= rank < world or world > P:
        raise ValueError("need 0 <= rank < world <= P")
    return rank * P // world, (rank + 1) * P // world


def merge_topk(parts, k: int):
    """Merge per-rank top-k lists (i, j, w arrays) into the global top-k,
    ordered by |w| descending, then i, then j ascending."""
    i = np.concatenate([np.asarray(p[0], np.int64) for p in parts]) if parts else np.zeros(0, np.int64)
    j = np.concatenate([np.asarray(p[1], np.int64) for p in parts]) if parts else np.zeros(0, np.int64)
    w = np.concatenate([np.asarray(p[2], np.float64) for p in parts]) if parts else np.zeros(0)
    order = np.lexsort((j, i, -np.abs(w)))[:k]
    return i[order], j[order], w[order]


def gather_topk(local, k: int, group=None):
    """All ranks pass their own top-k (i, j, w); rank 0 gets the global top-k,
    the others None.  Uses torch.distributed (gloo or nccl)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    payload = [np.asarray(x).tolist() for x in local]
    out = [None] * world
    dist.all_gather_object(out, payload, group=group)
    if dist.get_rank(group) != 0:
        return None
    return merge_topk([tuple(np.asarray(x) for x in o) for o in out], k)


def gather_sketch(local, group=None):
    """All ranks pass the P estimators of their interval plan's Count-Sketch
    (numpy int64 or float64, zero outside the interval); every rank gets the
    sketch of the whole product, their sum.  Uses torch.distributed."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(local)).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


def job_rate(units_total: float, ms_local: float, group=None) -> tuple[float, float]:
    """Whole-job throughput of a strong-scaling run: the ranks split one fixed
    product (each enumerates only its own partition interval, so the product's
    terms are counted once, not once per rank), and the job takes as long as
    its slowest rank.  Returns (units_total / slowest time in s, slowest time
    in ms); without an initialised process group, the local figures."""
    ms = float(ms_local)
    try:
        import torch.distributed as dist
        active = dist.is_available() and dist.is_initialized()
    except Exception:
        active = False
    if active:
        import torch
        backend = dist.get_backend(group)
        dev = "cuda" if backend == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        ms = float(t.item())
    return units_total / (ms / 1e3), ms
