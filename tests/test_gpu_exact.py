"""GPU parity of the exact column-row product against the CPU oracle.

Every test drives the CUDA path through the C ABI (ctypes binding) and
compares with the oracle on the same seeded inputs: integer counts bit-exact,
real values within 1e-6 relative of the fp64 oracle (the bound stated for the
compensated fp32 path)."""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O

pytestmark = pytest.mark.gpu

RTOL_REAL = 1e-6


@pytest.fixture(scope="module")
def crp():
    import torch
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp as c
    torch.cuda.init()
    return c


def _sorted(i, j, w):
    o = np.lexsort((j, i))
    return i[o].astype(np.int64), j[o].astype(np.int64), w[o]


def _run(crp, A, B, n_rows, n_cols, P, mode=O.FULL, value_type=0, **kw):
    dA = crp.to_device(A)
    dB = dA if B is A else crp.to_device(B)
    plan = crp.Plan(n_rows, n_cols, P, ci.SEED_A, ci.SEED_B, value_type=value_type, mode=mode,
                    flags=kw.pop("flags", crp.CRP_PLAN_DEBUG_CHECKS), **kw)
    plan.accumulate(dA, dB)
    plan.sync()
    return plan


def _check_exact(crp, plan, ref, P):
    i, j, w, _ = plan.export()
    gi, gj, gw = _sorted(i, j, w)
    assert np.array_equal(gi, ref.i) and np.array_equal(gj, ref.j)
    assert np.array_equal(gw, ref.w)
    # every entry sits in the partition h(i, j) and in no other
    for p in range(0, P, max(1, P // 8)):
        pi, pj, _, _ = plan.export(p, p + 1)
        assert (O.partition_of(pi, pj, P, ci.SEED_A, ci.SEED_B) == p).all()
    st = plan.stats(per_partition=True)
    assert st["terms"] == ref.terms
    assert st["entries"] == len(ref.i)
    return st


CONFIGS = [
    dict(groups=1), dict(groups=4), dict(groups=64, tile_vectors=16),
    dict(groups=1, smem_slots=4096, flags=0), dict(groups=16, smem_slots=16384, tile_vectors=256),
    dict(groups=2, flags=1 | 2),  # no warp match
    dict(flags=4 | 2), dict(groups=8, flags=4 | 2),  # direct HBM updates
    dict(flags=8 | 2), dict(groups=16, flags=8 | 2), dict(groups=64, flags=8 | 1 | 2),  # routed
    dict(flags=4 | 2, hot_items=64), dict(flags=4 | 2, hot_items=1000),  # direct + hot block
    dict(groups=16, flags=8 | 2, hot_items=128),                         # routed + hot block
    dict(flags=4 | 2, hot_items=64, warm_items=16),                      # direct + hot + warm
    dict(flags=4 | 2, warm_items=100),                                   # direct + warm only
    dict(groups=16, flags=8 | 2, hot_items=32, warm_items=128),          # routed, warm > hot
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_c1_cooccurrence_full_bit_exact(crp, cfg):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    cfg = dict(cfg)
    plan = _run(crp, T, T, 1000, 1000, 64, **cfg)
    st = _check_exact(crp, plan, ref, 64)
    want = O.partition_term_counts(Tc, Tc, 64, ci.SEED_A, ci.SEED_B)
    assert st["partition_terms"].astype(np.int64).tolist() == want.tolist()
    assert st["terms"] == int((T.lengths() ** 2).sum())
    plan.close()


@pytest.mark.parametrize("cfg", [dict(groups=8), dict(flags=4 | 16 | 2),
                                 dict(flags=8 | 16 | 2, hot_items=64),
                                 dict(flags=8 | 16 | 2, hot_items=64, warm_items=32)],
                         ids=["groups", "direct-sorted-rows", "routed-sorted-rows",
                              "routed-sorted-rows-warm"])
def test_c1_upper_and_topk(crp, cfg):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.UPPER)
    plan = _run(crp, T, T, 1000, 1000, 64, mode=O.UPPER, **cfg)
    _check_exact(crp, plan, ref, 64)
    assert ref.terms == int((T.lengths() * (T.lengths() - 1) // 2).sum())
    for k in (1, 10, 1000, 5000):
        ti, tj, tw, _ = plan.topk(k)
        ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k)
        assert np.array_equal(ti, ri) and np.array_equal(tj, rj) and np.array_equal(tw, rw)
    plan.close()


def test_topk_full_mode_upper_flag_and_large_k(crp):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = _run(crp, T, T, 1000, 1000, 64, groups=2)
    for k, up in ((1000, True), (8192, True), (8192, False), (3, False)):
        ti, tj, tw, _ = plan.topk(k, upper=up)
        ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k, upper_only=up)
        assert np.array_equal(ti, ri) and np.array_equal(tj, rj) and np.array_equal(tw, rw)
    # device outputs
    import torch
    ti, tj, tw, _ = plan.topk(100, upper=True, device_out="cuda")
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, 100, upper_only=True)
    assert np.array_equal(ti.cpu().numpy(), ri) and np.array_equal(tw.cpu().numpy(), rw)
    plan.close()


@pytest.mark.parametrize("cap", [1 << 21, 1 << 27])
def test_topk_sampled_histogram_on_large_tables(crp, cap):
    # tables of 2^26 slots or more take the top-k threshold from a 1/32 sample
    # histogram (falling back to the exact one when the sample is too thin);
    # the result must be the exact top k either way
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = _run(crp, T, T, 1000, 1000, 64, groups=1, flags=4 | 2, capacity_hint=cap)
    assert plan.stats()["table_slots"] >= cap
    for k, up in ((1, True), (10, False), (1000, True), (5000, False), (8192, True)):
        ti, tj, tw, _ = plan.topk(k, upper=up)
        ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k, upper_only=up)
        assert np.array_equal(ti, ri) and np.array_equal(tj, rj) and np.array_equal(tw, rw)
    plan.close()


def _random_case(seed, K, n_i, n_j, density, values):
    rng = np.random.default_rng(seed)
    ptrs, idxs = [], []
    for n in (n_i, n_j):
        ptr = [0]
        idx = []
        for k in range(K):
            r = rng.random()
            L = 0 if r < 0.1 else (1 if r < 0.2 else (n if r < 0.22 else rng.binomial(n, density)))
            idx.extend(np.sort(rng.choice(n, L, replace=False)).tolist())
            ptr.append(len(idx))
        ptrs.append(np.array(ptr, np.int64))
        idxs.append(np.array(idx, np.int32))
    vA = rng.uniform(0.01, 3, len(idxs[0])).astype(np.float32) if values else None
    vB = rng.uniform(0.01, 3, len(idxs[1])).astype(np.float32) if values else None
    A = O.Compressed(ptrs[0], idxs[0], vA, n_i)
    B = O.Compressed(ptrs[1], idxs[1], vB, n_j)
    return A, B


@pytest.mark.parametrize("seed,P,G,fl,hot,warm", [
    (0, 1, 1, 2, 0, 0), (1, 2, 2, 2, 0, 0), (2, 64, 8, 2, 0, 0), (3, 1024, 32, 2, 0, 0),
    (4, 4096, 4096, 2, 0, 0), (5, 16, 1, 2, 0, 0), (6, 256, 256, 8 | 2, 0, 0),
    (7, 1, 1, 8 | 2, 0, 0), (8, 64, 1, 4 | 2, 16, 0), (9, 16, 1, 4 | 2, 500, 0),
    (14, 64, 1, 4 | 2, 8, 40), (15, 32, 4, 8 | 2, 0, 4000), (16, 1, 1, 8 | 2, 3, 3)])
def test_random_edge_cases_int(crp, seed, P, G, fl, hot, warm):
    # warm=4000 exceeds both dimensions (the plan clamps it to min(n_rows, n_cols))
    A, B = _random_case(seed, 700, 37 + seed * 50, 53 + seed * 30, 0.2, False)
    ref = O.exact_product(A, B, O.FULL)
    plan = _run(crp, A, B, A.n_minor, B.n_minor, P, groups=G, tile_vectors=7, flags=fl,
                hot_items=hot, warm_items=warm)
    _check_exact(crp, plan, ref, P)
    plan.close()


@pytest.mark.parametrize("seed,G,fl", [(10, 1, 2), (11, 8, 2), (12, 4, 8 | 2), (13, 1, 4 | 2)])
def test_random_real_within_tolerance(crp, seed, G, fl):
    A, B = _random_case(seed, 600, 80, 90, 0.15, True)
    ref = O.exact_product(A, B, O.FULL)
    plan = _run(crp, A, B, 80, 90, 32, value_type=1, groups=G, flags=fl)
    i, j, w, _ = plan.export()
    gi, gj, gw = _sorted(i, j, w)
    assert np.array_equal(gi, ref.i) and np.array_equal(gj, ref.j)
    np.testing.assert_allclose(gw, ref.w, rtol=RTOL_REAL, atol=0)
    plan.close()


def test_real_single_product_entries_bit_exact(crp):
    # Every column of A holds one nonzero, so each entry of A A is one product:
    # the GPU's TwoProduct (p + e) must reproduce the fp64 product exactly.
    rng = np.random.default_rng(3)
    n = 3000
    rows = rng.integers(0, n, n).astype(np.int32)
    vals = rng.uniform(0.001, 1, n).astype(np.float32)
    A = O.Compressed(np.arange(n + 1, dtype=np.int64), rows, vals, n)
    At = O.Compressed.of(ci.transpose(ci.Sparse(A.ptr, A.idx, A.val, n)))
    ref = O.exact_product(A, At, O.FULL)
    plan = _run(crp, A, At, n, n, 16, value_type=1, groups=4)
    i, j, w, _ = plan.export()
    gi, gj, gw = _sorted(i, j, w)
    assert np.array_equal(gi, ref.i) and np.array_equal(gj, ref.j)
    assert np.array_equal(gw, ref.w)
    plan.close()


@pytest.mark.parametrize("fl", [2, 8 | 2])
def test_c3_markov_expansion_scaled(crp, fl):
    A, At = ci.c3(n=20_000, cmax=400)
    Ac, Atc = O.Compressed.of(A), O.Compressed.of(At)
    ref = O.exact_product(Ac, Atc, O.FULL)
    plan = _run(crp, A, At, A.n_minor, At.n_minor, 256, value_type=1, groups=16, flags=fl)
    i, j, w, _ = plan.export()
    gi, gj, gw = _sorted(i, j, w)
    assert np.array_equal(gi, ref.i) and np.array_equal(gj, ref.j)
    np.testing.assert_allclose(gw, ref.w, rtol=RTOL_REAL, atol=0)
    # column-stochastic A: A A is column-stochastic too
    colsum = np.bincount(gj, weights=gw, minlength=A.n_minor)
    has = np.bincount(gj, minlength=A.n_minor) > 0
    assert np.abs(colsum[has] - 1).max() < 1e-5
    ti, tj, tw, _ = plan.topk(500)
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, 500)
    np.testing.assert_allclose(tw, rw, rtol=RTOL_REAL)
    plan.close()


@pytest.mark.parametrize("cfg", [dict(groups=4, flags=2),
                                 dict(groups=16, flags=8 | 2, hot_items=64, warm_items=32),
                                 dict(flags=4 | 2, warm_items=48)],
                         ids=["groups", "routed+hot+warm", "direct+warm"])
def test_streaming_chunks_are_additive(crp, cfg):
    # each call picks its own hot / warm items and leaves the dense tiers clear
    T = ci.C1.scaled(m=9000).generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, **cfg)
    for lo, hi in ((0, 1000), (1000, 1001), (1001, 6000), (6000, 9000)):
        ptr = T.ptr[lo:hi + 1] - T.ptr[lo]
        part = ci.Sparse(ptr, T.idx[T.ptr[lo]:T.ptr[hi]], None, 1000)
        d = crp.to_device(part)
        plan.accumulate(d, d)
    plan.sync()
    _check_exact(crp, plan, ref, 64)
    plan.close()


def test_table_full_reported_and_auto_grow(crp):
    T = ci.C1.scaled(m=5000).generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    d = crp.to_device(T)
    plan = crp.Plan(1000, 1000, 16, ci.SEED_A, ci.SEED_B, capacity_hint=16 * 256)
    plan.accumulate(d, d)
    with pytest.raises(crp.CrpError) as e:
        plan.sync()
    assert e.value.status == crp.CRP_ETABLE_FULL
    plan.close()
    plan = crp.Plan(1000, 1000, 16, ci.SEED_A, ci.SEED_B, capacity_hint=16 * 256, auto_grow=True)
    plan.accumulate(d, d)
    plan.sync()
    assert plan.stats()["full_partitions"] == 0
    _check_exact(crp, plan, ref, 16)
    plan.close()


def test_invalid_arguments(crp):
    with pytest.raises(crp.CrpError) as e:
        crp.Plan(10, 10, 48, 1, 2)
    assert e.value.status == crp.CRP_EINVAL
    with pytest.raises(crp.CrpError):
        crp.Plan(10, 10, 64, 1, 2, groups=128)
    with pytest.raises(crp.CrpError):
        crp.Plan(0, 10, 64, 1, 2)
    plan = crp.Plan(100, 100, 4, 1, 2, flags=crp.CRP_PLAN_DEBUG_CHECKS)
    bad = ci.Sparse(np.array([0, 2], np.int64), np.array([3, 150], np.int32), None, 100)
    d = crp.to_device(bad)
    with pytest.raises(crp.CrpError) as e:
        plan.accumulate(d, d)
    assert e.value.status == crp.CRP_EINVAL
    vals = ci.Sparse(np.array([0, 1], np.int64), np.array([3], np.int32),
                     np.array([1.0], np.float32), 100)
    dv = crp.to_device(vals)
    with pytest.raises(crp.CrpError) as e:
        plan.accumulate(dv, dv)          # {0,1} plan given values
    assert e.value.status == crp.CRP_EINVAL
    plan.close()


def test_partition_of_matches_oracle(crp):
    plan = crp.Plan(10**6, 10**6, 8192, ci.SEED_A, ci.SEED_B, capacity_hint=8192 * 64)
    rng = np.random.default_rng(0)
    i = rng.integers(0, 10**6, 300)
    j = rng.integers(0, 10**6, 300)
    want = O.partition_of(i, j, 8192, ci.SEED_A, ci.SEED_B)
    assert [plan.partition_of(int(a), int(b)) for a, b in zip(i, j)] == want.tolist()
    plan.close()


@pytest.mark.parametrize("cfg", [dict(groups=16, flags=8 | 2, hot_items=64, warm_items=16),
                                 dict(flags=4 | 2), dict(groups=4, flags=2)],
                         ids=["routed", "direct", "smem"])
def test_reset_between_calls(crp, cfg):
    # a reset empties the tables before anything reads them again (the routed
    # path runs it beside its routing kernel): reset -> empty top-k and
    # stats; reset -> accumulate -> the product; two calls -> twice it
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    d = crp.to_device(T)
    plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, **cfg)
    plan.accumulate(d, d)
    plan.sync()
    _check_exact(crp, plan, ref, 64)
    plan.reset()
    assert len(plan.topk(10)[0]) == 0
    assert plan.stats()["entries"] == 0
    plan.accumulate(d, d)
    plan.sync()
    _check_exact(crp, plan, ref, 64)
    plan.reset()
    plan.accumulate(d, d)
    plan.accumulate(d, d)
    plan.sync()
    i, j, w, _ = plan.export()
    gi, gj, gw = _sorted(i, j, w)
    assert np.array_equal(gi, ref.i) and np.array_equal(gj, ref.j)
    assert np.array_equal(gw, 2 * ref.w)
    plan.reset()
    plan.accumulate(d, d)
    plan.sync()
    _check_exact(crp, plan, ref, 64)
    plan.close()


def test_repeat_runs_bit_identical(crp):
    T = ci.C1.scaled(m=8000).generate()
    d = crp.to_device(T)
    outs = []
    for G in (1, 8, 1):
        plan = crp.Plan(1000, 1000, 64, ci.SEED_A, ci.SEED_B, groups=G)
        plan.accumulate(d, d)
        plan.sync()
        outs.append(_sorted(*plan.export()[:3]))
        plan.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("cfg", [dict(flags=4 | 2), dict(flags=4 | 2, hot_items=256),
                                 dict(groups=16, flags=2), dict(groups=1, flags=2),
                                 dict(groups=32, flags=8 | 2, hot_items=128),
                                 dict(groups=32, flags=8 | 2, hot_items=64, warm_items=64)],
                         ids=["direct", "direct+hot", "lemma1-groups", "smem", "routed+hot",
                              "routed+hot+warm"])
def test_disjoint_intervals_union_is_the_product(crp, cfg):
    # Figure 1 / Theorem 1: K instances of CRoP on disjoint intervals of the
    # partitions, each seeing the whole input, together produce every entry
    # exactly once, and each keeps only the entries hashing into its interval.
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    P = 64
    d = crp.to_device(T)
    got_i, got_j, got_w = [], [], []
    for q, r in ((0, 16), (16, 48), (48, 64)):
        plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, part_begin=q, part_end=r, **cfg)
        plan.accumulate(d, d)
        plan.sync()
        i, j, w, _ = plan.export()
        p = O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B)
        assert ((p >= q) & (p < r)).all()
        got_i.append(i)
        got_j.append(j)
        got_w.append(w)
        plan.close()
    i, j, w = map(np.concatenate, (got_i, got_j, got_w))
    gi, gj, gw = _sorted(i, j, w)
    assert np.array_equal(gi, ref.i) and np.array_equal(gj, ref.j) and np.array_equal(gw, ref.w)


@pytest.mark.parametrize("pool", [1, 3000], ids=["one-chunk", "3000-chunks"])
def test_routed_pool_exhaustion_paths(crp, pool):
    """The routed pool capped below the records it needs (route_pool_chunks):
    appends that find the pool dry go to the overflow chunks (256 chunks of
    512 records here) and, once those fill, straight to the tables; the
    product stays bit-exact.  pool = 1 leaves one chunk besides the overflow
    chunks; 3000 leaves about one per (CTA, bin), so it runs dry part way."""
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    for hot, warm in ((0, 0), (64, 16)):
        plan = _run(crp, T, T, 1000, 1000, 64, groups=16, flags=8 | 2, hot_items=hot,
                    warm_items=warm, route_pool_chunks=pool)
        _check_exact(crp, plan, ref, 64)
        plan.close()


@pytest.mark.parametrize("w,P,tol", [(ci.C2.scaled(m=300_000), 1024, 0.02),
                                     (ci.C2.scaled(m=100_000), 256, 0.05)],
                         ids=["300k-tx-P1024", "100k-tx-P256"])
def test_distinct_count_estimate_against_the_oracle(crp, w, P, tol):
    """The tables are sized from an estimate of the product's distinct
    entries: the entries of the partitions [0, P / G) (G = min(P, 64) groups)
    counted exactly on the GPU, times G.  h is pairwise independent, so each
    group holds ~1/G of the entries; against the oracle's exact count the
    estimate is within `tol` (a few standard deviations of the sampled share:
    16 partitions of ~40,000 entries, or 4 of ~60,000).  (Products with at
    most 2^22 possible entries are not sampled: their tables are sized from
    the bound.)"""
    T = w.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    d = crp.to_device(T)
    plan = crp.Plan(T.n_minor, T.n_minor, P, ci.SEED_A, ci.SEED_B, flags=4, auto_grow=True)
    plan.accumulate(d, d)
    plan.sync()
    st = plan.stats()
    assert st["entries"] == len(ref.i)
    est = st["estimated_entries"]
    assert est > 0
    assert abs(est - len(ref.i)) <= tol * len(ref.i), (est, len(ref.i))
    plan.close()


@pytest.mark.parametrize("hot,warm", [(512, 200), (300, 128), (129, 129), (2048, 64)],
                         ids=["warm-above-core", "warm-equal-core", "hot-just-above-core",
                              "hot2048-warm64"])
def test_routed_class_sorted_walk_tier_orders(crp, hot, warm):
    """The routed walk orders each staged side by dense-tier class; the
    rectangles it walks depend on whether the warm width is below, at or
    above the 128-item shared-memory core.  Every order gives the oracle's
    product exactly (Zipf(1.1) transactions over 1,000 items, so the tiers hold
    most items)."""
    T = ci.C1.scaled(m=20_000).generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    plan = _run(crp, T, T, T.n_minor, T.n_minor, 64,
                flags=crp.CRP_PLAN_ROUTED | crp.CRP_PLAN_DEBUG_CHECKS, groups=0,
                hot_items=hot, warm_items=warm)
    _check_exact(crp, plan, ref, 64)
    plan.close()
