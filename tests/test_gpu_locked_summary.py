"""GPU locked-bucket summaries (CRP_PLAN_LOCKED_SUMMARY): each partition is one
Space-Saving summary of exactly ell counters updated under a lock, the
paper's regime of many buckets with two counters (Section 6).

The lock serialises the updates of a bucket, so each bucket is the
sequential algorithm of the Preliminaries run on one arrival order of its
partition's terms.  Which order is not fixed, so the tests check what every
order gives, against the exact product from the oracle: at most ell keys per
partition; the counts of a bucket sum to the partition's weight W_p exactly
(each weighted update adds its weight to exactly one counter); lower <= true
<= upper for every recorded key; every overestimation <= the bucket's
smallest count <= W_p / ell; every key heavier than W_p / ell recorded; a
partition with at most ell distinct keys exact (tests/summary_checks.py;
the oracle's sequential Space-Saving passes the same checks)."""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O
from summary_checks import _check_buckets, _truth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crp():
    import torch
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp as c
    torch.cuda.init()
    return c


CONFIGS = [
    dict(P=64, ell=2), dict(P=1024, ell=2), dict(P=64, ell=1), dict(P=256, ell=3),
    dict(P=16, ell=8), dict(P=4096, ell=2, groups=16),
    dict(P=1024, ell=2, flags=4),                        # direct: every term takes a lock
    dict(P=1024, ell=2, flags=4, hot_items=64, warm_items=8),   # dense tiers, weighted at the end
    dict(P=1024, ell=2, flags=4 | 1),                    # direct without warp pre-combining
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_c1_locked_buckets(crp, cfg):
    cfg = dict(cfg)
    P, ell = cfg.pop("P"), cfg.pop("ell")
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref, part, true, W, distinct = _truth(Tc, Tc, P)
    flags = crp.CRP_PLAN_LOCKED_SUMMARY | crp.CRP_PLAN_DEBUG_CHECKS | cfg.pop("flags", 0)
    plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, summary_counters=ell, flags=flags, **cfg)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    i, j, up, lo = plan.export()
    _check_buckets(i, j, up, lo, P, ell, 1000, true, W, distinct, ref, part)
    st = plan.stats()
    assert st["terms"] == ref.w.sum()
    # top-k ranks the recorded keys by their upper bound
    ti, tj, tw, tl = plan.topk(100)
    o = np.lexsort((j, i, -up))[:100]
    assert np.array_equal(tw, up[o]) and np.array_equal(tl, lo[o])
    plan.close()


def test_c1_upper_sorted_rows(crp):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    P, ell = 512, 2
    ref, part, true, W, distinct = _truth(Tc, Tc, P, O.UPPER)
    plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER, summary_counters=ell,
                    flags=crp.CRP_PLAN_LOCKED_SUMMARY | crp.CRP_PLAN_SORTED_ROWS |
                    crp.CRP_PLAN_DIRECT, hot_items=32, warm_items=4)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    i, j, up, lo = plan.export()
    assert (i < j).all()
    _check_buckets(i, j, up, lo, P, ell, 1000, true, W, distinct, ref, part)
    plan.close()


def test_streaming_reset_and_sketch(crp):
    # two calls give the invariants of the whole stream; the sketch beside
    # the buckets is exact; reset empties both
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    P, ell = 256, 2
    ref, part, true, W, distinct = _truth(Tc, Tc, P)
    plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, summary_counters=ell,
                    flags=crp.CRP_PLAN_LOCKED_SUMMARY | crp.CRP_PLAN_SKETCH)
    m = T.n_major // 2
    for lo_, hi_ in ((0, m), (m, T.n_major)):
        sub = ci.Sparse(T.ptr[lo_:hi_ + 1] - T.ptr[lo_], T.idx[T.ptr[lo_]:T.ptr[hi_]], None, 1000)
        dd = crp.to_device(sub)
        plan.accumulate(dd, dd)
    plan.sync()
    i, j, up, lo = plan.export()
    _check_buckets(i, j, up, lo, P, ell, 1000, true, W, distinct, ref, part)
    assert np.array_equal(plan.sketch(), O.count_sketch(ref, P, ci.SEED_A, ci.SEED_B))
    plan.reset()
    assert len(plan.export()[0]) == 0 and not plan.sketch().any()
    plan.close()


@pytest.mark.parametrize("seed,P,ell,fl", [(0, 1, 2, 0), (1, 2, 1, 4), (2, 8, 4, 0), (3, 64, 2, 4),
                                           (4, 1, 3, 4)])
def test_random_edge_cases(crp, seed, P, ell, fl):
    # P = 1: every update waits for the same lock
    rng = np.random.default_rng(seed)
    out = []
    for n in (50, 60):
        ptr, idx = [0], []
        for _ in range(300):
            r = rng.random()
            L = 0 if r < 0.1 else (1 if r < 0.2 else (n if r < 0.22 else rng.binomial(n, 0.2)))
            idx.extend(np.sort(rng.choice(n, L, replace=False)).tolist())
            ptr.append(len(idx))
        out.append(O.Compressed(np.array(ptr, np.int64), np.array(idx, np.int32), None, n))
    A, B = out
    ref, part, true, W, distinct = _truth(A, B, P)
    plan = crp.Plan(50, 60, P, ci.SEED_A, ci.SEED_B, summary_counters=ell,
                    flags=crp.CRP_PLAN_LOCKED_SUMMARY | crp.CRP_PLAN_DEBUG_CHECKS | fl)
    plan.accumulate(crp.to_device(A), crp.to_device(B))
    plan.sync()
    i, j, up, lo = plan.export()
    _check_buckets(i, j, up, lo, P, ell, 60, true, W, distinct, ref, part)
    plan.close()


def test_invalid_locked_plans_are_rejected(crp):
    F = crp.CRP_PLAN_LOCKED_SUMMARY
    for kw in (dict(summary_counters=0), dict(summary_counters=65),
               dict(summary_counters=2, reserved_counters=16),
               dict(summary_counters=2, flags=F | crp.CRP_PLAN_ROUTED),
               dict(summary_counters=2, hot_items=16)):      # dense tiers need the direct kernel
        kw.setdefault("flags", F)
        with pytest.raises(crp.CrpError):
            crp.Plan(100, 100, 16, 1, 2, **kw)


@pytest.mark.parametrize("flags", [0, 4], ids=["on-chip-table", "direct"])
def test_lock_wait_runs_out_and_the_plan_recovers(crp, flags):
    """A bucket lock that is never handed on (taken on the host through
    crp_debug_hold_lock, a failure injected without a GPU fault): the waits
    for it give up after lock_wait_us, crp_sync reports CRP_ETIMEOUT, and
    after crp_reset the same plan runs the product with every bucket check
    passing (the context stays usable)."""
    import time
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    # P = 1024 buckets and a 200 ms bound: without the held lock no wait
    # comes near the bound (with few buckets and a lock per term, the queue
    # on one bucket can legitimately take tens of ms)
    P, ell = 1024, 2
    ref, part, true, W, distinct = _truth(Tc, Tc, P)
    plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, summary_counters=ell,
                    flags=crp.CRP_PLAN_LOCKED_SUMMARY | flags, lock_wait_us=200_000)
    d = crp.to_device(T)
    plan.debug_hold_lock(5)
    t0 = time.time()
    plan.accumulate(d, d)
    with pytest.raises(crp.CrpError) as e:
        plan.sync()
    assert e.value.status == crp.CRP_ETIMEOUT
    assert time.time() - t0 < 30
    plan.reset()
    plan.accumulate(d, d)
    plan.sync()
    i, j, up, lo = plan.export()
    _check_buckets(i, j, up, lo, P, ell, 1000, true, W, distinct, ref, part)
    with pytest.raises(crp.CrpError) as e:
        plan.debug_hold_lock(P)
    assert e.value.status == crp.CRP_EINVAL
    plan.close()
