"""GPU summary mode (per-partition counters with Space-Saving guarantees)
against the exact oracle and the sequential Space-Saving oracle.

Several summaries are correct (the GPU merges exact window aggregates, the
sequential algorithm replaces one minimum at a time), so the tests check what
the paper fixes for Space-Saving (Preliminaries): lower <= true <= upper,
upper - lower <= W/ell, every key heavier than W/ell recorded, at most ell
keys per partition; exactness when ell covers every key; reserved keys exact."""
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


def _truth(T, P, mode=O.FULL):
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, mode)
    part = O.partition_of(ref.i, ref.j, P, ci.SEED_A, ci.SEED_B)
    true = dict(zip((ref.i * T.n_minor + ref.j).tolist(), ref.w.tolist()))
    W = np.bincount(part, weights=ref.w, minlength=P)
    return ref, true, W


def _summary_plan(crp, T, P, ell, reserved=0, mode=O.FULL, flags=0):
    d = crp.to_device(T)
    plan = crp.Plan(T.n_minor, T.n_minor, P, ci.SEED_A, ci.SEED_B, mode=mode,
                    summary_counters=ell, reserved_counters=reserved, flags=flags)
    return plan, d


def test_summary_exact_when_counters_cover_every_key(crp):
    T = ci.C1.scaled(m=6000).generate()
    P = 16
    ref, true, W = _truth(T, P)
    per_part = np.bincount(O.partition_of(ref.i, ref.j, P, ci.SEED_A, ci.SEED_B), minlength=P)
    plan, d = _summary_plan(crp, T, P, int(per_part.max()) + 1)
    plan.accumulate(d, d)
    plan.sync()
    i, j, w, wl = plan.export()
    o = np.lexsort((j, i))
    assert np.array_equal(i[o], ref.i) and np.array_equal(j[o], ref.j)
    assert np.array_equal(w[o], ref.w) and np.array_equal(wl[o], ref.w)
    plan.close()


@pytest.mark.parametrize("P,ell", [(16, 256), (64, 32), (4, 2048)])
def test_summary_space_saving_guarantees(crp, P, ell):
    T = ci.C1.generate()
    ref, true, W = _truth(T, P)
    plan, d = _summary_plan(crp, T, P, ell)
    plan.accumulate(d, d)
    plan.sync()
    for p in range(P):
        i, j, up, lo = plan.export(p, p + 1)
        keys = (i.astype(np.int64) * T.n_minor + j).tolist()
        assert len(keys) <= ell
        assert (O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B) == p).all()
        tv = np.array([true[k] for k in keys])
        assert (lo <= tv).all() and (tv <= up).all()
        assert ((up - lo) <= W[p] / ell + 1e-9).all()
        assert up.sum() <= W[p]
        got = set(keys)
        part_keys = np.flatnonzero(O.partition_of(ref.i, ref.j, P, ci.SEED_A, ci.SEED_B) == p)
        for q in part_keys[ref.w[part_keys] > W[p] / ell]:
            assert int(ref.i[q] * T.n_minor + ref.j[q]) in got
    plan.close()


def _weight_err(ti, tj, true, ref, k, n):
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k, upper_only=True)
    got = sum(true.get(int(a) * n + int(b), 0.0) for a, b in zip(ti, tj))
    return 1.0 - got / rw.sum()


def test_summary_topk_weight_error_vs_sequential_space_saving(crp):
    T = ci.C1.generate()
    P, ell, k = 16, 128, 200
    ref, true, W = _truth(T, P)
    plan, d = _summary_plan(crp, T, P, ell)
    plan.accumulate(d, d)
    plan.sync()
    ti, tj, tw, tl = plan.topk(k, upper=True)
    gpu_err = _weight_err(ti, tj, true, ref, k, T.n_minor)
    # sequential Space-Saving per partition (the oracle's reading of Figure 1)
    streams = O.partition_streams(O.Compressed.of(T), O.Compressed.of(T), P, ci.SEED_A,
                                  ci.SEED_B, O.FULL)
    cand = []
    for s in streams:
        for key, (c, o) in O.space_saving(s, ell).items():
            cand.append((key // T.n_minor, key % T.n_minor, c))
    ci_, cj_, cw_ = map(np.array, zip(*cand))
    si, sj, _ = O.topk(ci_, cj_, cw_, k, upper_only=True)
    seq_err = _weight_err(si, sj, true, ref, k, T.n_minor)
    assert gpu_err <= seq_err + 0.02, (gpu_err, seq_err)
    # the bounds of the reported heavy entries
    for a, b, u, l in zip(ti, tj, tw, tl):
        assert l <= true[int(a) * T.n_minor + int(b)] <= u
    plan.close()


def test_reserved_keys_are_counted_exactly(crp):
    T = ci.C1.generate()
    P, ell = 16, 64
    ref, true, W = _truth(T, P)
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, 300, upper_only=True)
    keys = (ri.astype(np.uint64) << np.uint64(32)) | rj.astype(np.uint64)
    plan, d = _summary_plan(crp, T, P, ell, reserved=1024)
    plan.reserve(keys)
    for rep in range(2):   # reset keeps the reserved keys
        plan.accumulate(d, d)
        plan.sync()
        # P * ell summary keys + 300 reserved keys < 8192: top-k returns all
        ti, tj, tw, tl = plan.topk(8192)
        got = {(int(a), int(b)): (u, l) for a, b, u, l in zip(ti, tj, tw, tl)}
        for a, b, w in zip(ri, rj, rw):
            assert got[(int(a), int(b))] == (w, w)
        assert len(ti) <= P * ell + 300
        plan.reset()
    plan.close()


def test_reserved_dense_block_keeps_guarantees(crp):
    # the rows and columns of the reserved keys index a dense block whose
    # reserved cells count those pairs during the call (the other pairs of the
    # block take the summary path) and go to the exact counters at its end:
    # the reserved counts are exact and every summary entry keeps the
    # Space-Saving bounds, over two streaming calls
    T = ci.C1.scaled(m=12000).generate()
    P, ell = 8, 128
    ref, true, W = _truth(T, P)
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, 200, upper_only=False)
    keys = (ri.astype(np.uint64) << np.uint64(32)) | rj.astype(np.uint64)
    plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, summary_counters=ell,
                    reserved_counters=256)
    plan.reserve(keys)
    for lo, hi in ((0, 5000), (5000, 12000)):
        part = ci.Sparse(T.ptr[lo:hi + 1] - T.ptr[lo], T.idx[T.ptr[lo]:T.ptr[hi]], None, 1000)
        dd = crp.to_device(part)
        plan.accumulate(dd, dd)
    plan.sync()
    reserved = set((int(a) * 1000 + int(b)) for a, b in zip(ri, rj))
    i, j, up, lo_ = plan.export()   # the summaries (reserved counters are not in them)
    kk = (i.astype(np.int64) * 1000 + j)
    assert not any(int(k) in reserved for k in kk)
    tv = np.array([true[int(k)] for k in kk])
    assert (lo_ <= tv).all() and (tv <= up).all()
    p = O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B)
    assert ((up - lo_) <= W[p] / ell + 1e-9).all()
    # P * ell summary keys + 200 reserved keys < 8192: top-k returns all
    ti, tj, tw, tl = plan.topk(8192)
    got = {(int(a), int(b)): (u, l) for a, b, u, l in zip(ti, tj, tw, tl)}
    for a, b, w in zip(ri, rj, rw):
        assert got[(int(a), int(b))] == (w, w)
    plan.close()


def test_summary_streaming_chunks_keep_guarantees(crp):
    T = ci.C1.scaled(m=12000).generate()
    P, ell = 8, 256
    ref, true, W = _truth(T, P)
    plan = crp.Plan(1000, 1000, P, ci.SEED_A, ci.SEED_B, summary_counters=ell)
    for lo, hi in ((0, 3000), (3000, 3001), (3001, 12000)):
        part = ci.Sparse(T.ptr[lo:hi + 1] - T.ptr[lo], T.idx[T.ptr[lo]:T.ptr[hi]], None, 1000)
        dd = crp.to_device(part)
        plan.accumulate(dd, dd)
    plan.sync()
    i, j, up, lo_ = plan.export()
    keys = (i.astype(np.int64) * 1000 + j).tolist()
    tv = np.array([true[k] for k in keys])
    p = O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B)
    assert (lo_ <= tv).all() and (tv <= up).all()
    assert ((up - lo_) <= W[p] / ell + 1e-9).all()
    plan.close()


def test_summary_upper_sorted_rows_guarantees(crp):
    # pairs above the diagonal, enumerated only as j after i (sorted rows)
    T = ci.C1.generate()
    P, ell = 16, 128
    ref, true, W = _truth(T, P, O.UPPER)
    plan, d = _summary_plan(crp, T, P, ell, mode=O.UPPER, flags=crp.CRP_PLAN_SORTED_ROWS)
    plan.accumulate(d, d)
    plan.sync()
    i, j, up, lo = plan.export()
    assert (i < j).all()
    keys = (i.astype(np.int64) * T.n_minor + j).tolist()
    tv = np.array([true[k] for k in keys])
    p = O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B)
    assert (lo <= tv).all() and (tv <= up).all()
    assert ((up - lo) <= W[p] / ell + 1e-9).all()
    assert plan.stats()["terms"] == ref.terms
    plan.close()
