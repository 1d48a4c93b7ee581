"""Top-k answered from the hot block (crp_topk_certified_calls): for {0,1}
inputs an entry is at most the smaller degree of its row and column, so when
the k-th heaviest hot pair weighs more than every degree outside the hot set
the top k lies among the hot pairs.  The answer must equal the oracle's top k
whether the bound holds (answered from the hot pairs) or not (full scan),
including ties at the bound, streaming calls with different hot sets, and
partition intervals."""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crp():
    import torch
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp as c
    torch.cuda.init()
    return c


def _check(plan, ref, k, up):
    ti, tj, tw, tl = plan.topk(k, upper=up)
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k, upper_only=up)
    assert np.array_equal(ti, ri) and np.array_equal(tj, rj) and np.array_equal(tw, rw)
    assert np.array_equal(tl, tw)


@pytest.mark.parametrize("flags,hot,warm", [(8 | 2, 128, 16), (4 | 2, 1000, 0), (8 | 2, 16, 0),
                                            (4 | 2, 64, 32)])
def test_c1_topk_equals_oracle_with_or_without_the_bound(crp, flags, hot, warm):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, flags=flags, hot_items=hot,
                    warm_items=warm)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    for k, up in ((1, True), (10, True), (100, False), (1000, True), (8192, False)):
        _check(plan, ref, k, up)
    if hot >= 128:   # the head of a Zipf(1.1) stream: the small k are certified
        assert plan.topk_certified_calls() >= 2
    plan.close()


def test_streaming_calls_with_different_hot_sets(crp):
    # degrees add up over the calls since the reset; the hot set is the last
    # call's; the two halves draw their heads from different items
    T1 = ci.C1.scaled(m=8000).generate()
    T2 = ci.transactions(ci.C1.seed + 77, 8000, 1000, 10.0, 2, 40, 1.1)
    # relabel the second half so its most frequent items differ
    T2 = ci.Sparse(T2.ptr, ((T2.idx.astype(np.int64) * 7 + 13) % 1000).astype(np.int32), None, 1000)
    rows = [np.sort(T2.idx[T2.ptr[k]:T2.ptr[k + 1]]) for k in range(T2.n_major)]
    T2 = ci.Sparse(T2.ptr, np.concatenate(rows).astype(np.int32), None, 1000)
    both = ci.Sparse(np.concatenate([T1.ptr, T2.ptr[1:] + T1.ptr[-1]]),
                     np.concatenate([T1.idx, T2.idx]), None, 1000)
    Bc = O.Compressed.of(both)
    ref = O.exact_product(Bc, Bc, O.FULL)
    plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, flags=8 | 2, hot_items=64)
    for part in (T1, T2):
        d = crp.to_device(part)
        plan.accumulate(d, d)
    plan.sync()
    for k, up in ((1, True), (20, True), (300, False), (2000, True)):
        _check(plan, ref, k, up)
    plan.reset()
    d = crp.to_device(T2)
    plan.accumulate(d, d)
    plan.sync()
    T2c = O.Compressed.of(T2)
    ref2 = O.exact_product(T2c, T2c, O.FULL)
    for k, up in ((1, True), (50, True)):
        _check(plan, ref2, k, up)
    plan.close()


def _tx(rows, n=10):
    ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    idx = np.concatenate([np.array(r, np.int32) for r in rows])
    return ci.Sparse(ptr, idx, None, n)


def test_bound_is_strict_at_ties(crp):
    # (0,1) and (2,3) both weigh 50 and items 2, 3 (outside the two hot items)
    # have degree 50: the k-th hot weight is not above the bound, so the
    # tables are scanned; the tie goes to (0,1) by (i, j)
    T = _tx([[0, 1]] * 50 + [[2, 3]] * 50 + [[0]] * 10 + [[1]] * 10)
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = crp.Plan(10, 10, 4, ci.SEED_A, ci.SEED_B, flags=8 | 2, hot_items=2)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    before = plan.topk_certified_calls()
    _check(plan, ref, 1, True)
    assert plan.topk_certified_calls() == before
    _check(plan, ref, 2, True)
    plan.close()
    # one more (0,1): now 51 > 50 and the top 1 is certified
    T = _tx([[0, 1]] * 51 + [[2, 3]] * 50 + [[0]] * 10 + [[1]] * 10)
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = crp.Plan(10, 10, 4, ci.SEED_A, ci.SEED_B, flags=8 | 2, hot_items=2)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    _check(plan, ref, 1, True)
    assert plan.topk_certified_calls() == 1
    _check(plan, ref, 2, True)          # one hot pair only: scanned
    assert plan.topk_certified_calls() == 1
    plan.close()


def test_partition_interval_plan(crp):
    # a plan owning part of the partitions: its top k is the top k of its
    # entries, however the hot pairs fall
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    keep = O.partition_of(ref.i, ref.j, 64, ci.SEED_A, ci.SEED_B) < 24
    sub = O.Product(ref.i[keep], ref.j[keep], ref.w[keep], int(ref.w[keep].sum()), ref.n_cols)
    plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, flags=8 | 2, hot_items=256,
                    part_begin=0, part_end=24)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    for k, up in ((1, True), (100, True), (1000, False)):
        _check(plan, sub, k, up)
    plan.close()


def test_separate_a_and_b_arrays_and_a_mix_of_calls(crp):
    # B given as other arrays than A (its degrees counted on their own), and
    # a first call with B == A followed by one with separate arrays
    T1 = ci.C1.scaled(m=9000).generate()
    T2 = ci.transactions(ci.C1.seed + 5, 9000, 1000, 10.0, 2, 40, 1.1)
    both = ci.Sparse(np.concatenate([T1.ptr, T2.ptr[1:] + T1.ptr[-1]]),
                     np.concatenate([T1.idx, T2.idx]), None, 1000)
    for calls in (((T2, False),), ((T1, True), (T2, False))):
        plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, flags=8 | 2, hot_items=100)
        for T, same in calls:
            a = crp.to_device(T)
            b = a if same else crp.to_device(T)
            plan.accumulate(a, b)
        plan.sync()
        src = T2 if len(calls) == 1 else both
        Sc = O.Compressed.of(src)
        ref = O.exact_product(Sc, Sc, O.FULL)
        before = plan.topk_certified_calls()
        for k, up in ((1, True), (10, True), (500, False)):
            _check(plan, ref, k, up)
        assert plan.topk_certified_calls() > before
        plan.close()
