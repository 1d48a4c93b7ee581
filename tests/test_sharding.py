"""Partition-interval sharding on CPU: two gloo ranks own disjoint intervals,
and the gathered top-k equals the top-k of the whole product (oracle)."""
import os
import socket

import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O
from paper_1210_0461_gb300.sharding import merge_topk, partition_interval


def test_intervals_cover_partitions_disjointly():
    for P, world in ((64, 2), (64, 3), (1024, 8), (8, 8)):
        iv = [partition_interval(r, world, P) for r in range(world)]
        assert iv[0][0] == 0 and iv[-1][1] == P
        assert all(a[1] == b[0] and a[0] < a[1] for a, b in zip(iv, iv[1:]))
    with pytest.raises(ValueError):
        partition_interval(0, 9, 8)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, P, k, out):
    import torch.distributed as dist
    from paper_1210_0461_gb300.sharding import gather_topk
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T = O.Compressed.of(ci.C1.scaled(m=4000).generate())
    full = O.exact_product(T, T, O.UPPER)
    q, r = partition_interval(rank, world, P)
    p = O.partition_of(full.i, full.j, P, ci.SEED_A, ci.SEED_B)
    mine = (p >= q) & (p < r)                      # this rank's instance of CRoP
    local = O.topk(full.i[mine], full.j[mine], full.w[mine], k)
    merged = gather_topk(local, k)
    if rank == 0:
        out.put([np.asarray(x).tolist() for x in merged])
    dist.barrier()
    dist.destroy_process_group()


def test_gathered_topk_equals_global_topk_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    P, k, world = 64, 50, 2
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, P, k, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    T = O.Compressed.of(ci.C1.scaled(m=4000).generate())
    full = O.exact_product(T, T, O.UPPER)
    want = O.topk(full.i, full.j, full.w, k)
    assert [list(map(float, x)) for x in got] == [list(map(float, x)) for x in want]


def test_merge_topk_ties_and_order():
    a = (np.array([1, 0]), np.array([2, 5]), np.array([7., 7.]))
    b = (np.array([0, 3]), np.array([1, 4]), np.array([7., 9.]))
    i, j, w = merge_topk([a, b], 3)
    assert list(zip(i, j, w)) == [(3, 4, 9.), (0, 1, 7.), (0, 5, 7.)]



def _sketch_worker(rank, world, port, P, out):
    import torch.distributed as dist
    from paper_1210_0461_gb300.sharding import gather_sketch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T = O.Compressed.of(ci.C1.scaled(m=4000).generate())
    full = O.exact_product(T, T, O.FULL)
    q, r = partition_interval(rank, world, P)
    local = O.count_sketch(full, P, ci.SEED_A, ci.SEED_B).astype(np.int64)
    local[:q] = 0
    local[r:] = 0                                   # this rank's interval plan
    merged = gather_sketch(local)
    out.put((rank, merged.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_gathered_sketch_equals_the_whole_sketch_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    P, world = 64, 2
    port = _free_port()
    procs = [ctx.Process(target=_sketch_worker, args=(r, world, port, P, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    T = O.Compressed.of(ci.C1.scaled(m=4000).generate())
    want = O.count_sketch(O.exact_product(T, T, O.FULL), P, ci.SEED_A, ci.SEED_B)
    for r in range(world):
        assert np.array_equal(np.array(got[r]), want)


def _rate_worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_1210_0461_gb300.sharding import job_rate
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 100 + 50 r ms for its interval of a 3e9-term product
    out.put((rank, job_rate(3e9, 100.0 + 50.0 * rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_counts_the_product_once_over_the_slowest_rank():
    """Strong scaling by partition interval: two ranks split one product of
    3e9 terms; the job's rate is 3e9 terms over the slower rank's 150 ms on
    every rank, not twice that."""
    import torch.multiprocessing as mp
    from paper_1210_0461_gb300.sharding import job_rate
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_rate_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for r in range(world):
        rate, ms = got[r]
        assert ms == 150.0
        assert rate == 3e9 / 0.150
    assert job_rate(3e9, 100.0) == (3e9 / 0.1, 100.0)     # one process, no group
