"""Parity at the full size of the 10,000,000-transaction x 100,000-item
co-occurrence workload, in the launch configuration bench.py times (routed,
bins sized by the plan, hot block of 2048 items, warm stripes of 32 or 64
items, the two widths the autotuner chooses between on this workload):
properties that hold at any size (every term stored exactly once, every
entry in its own partition, the diagonal equal to the item supports),
sampled entries -- present and absent -- computed one by one by the oracle
from the definition of an entry as an inner product, whole partitions
against the oracle's entries of that partition, and the top 1000 pairs
against the oracle's certified heaviest pairs of this input."""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O

pytestmark = pytest.mark.gpu

P = 1024


@pytest.fixture(scope="module", params=[32, 64], ids=["warm32", "warm64"])
def full(request):
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp
    T = ci.C2.generate()
    L = T.lengths().astype(np.int64)
    d = crp.to_device(T)
    plan = crp.Plan(T.n_minor, T.n_minor, P, ci.SEED_A, ci.SEED_B, groups=0,
                    flags=crp.CRP_PLAN_ROUTED, hot_items=2048, warm_items=request.param,
                    auto_grow=True)
    plan.accumulate(d, d)
    plan.sync()
    inv = O.Compressed.of(ci.transpose(T))   # item -> transactions (rows of A, columns of B)
    yield crp, T, L, plan, inv
    plan.close()


def test_every_term_stored_once(full):
    crp, T, L, plan, inv = full
    st = plan.stats(per_partition=True)
    total = int((L * L).sum())
    assert st["terms"] == total
    assert int(st["partition_terms"].astype(np.int64).sum()) == total
    assert st["spilled"] == 0 and st["full_partitions"] == 0


def test_sampled_partitions(full):
    crp, T, L, plan, inv = full
    rng = np.random.default_rng(2024)
    support = np.diff(inv.ptr)
    n = T.n_minor
    for p in rng.choice(P, 4, replace=False).tolist():
        i, j, w, _ = plan.export(p, p + 1)
        assert len(i) > 0
        i, j = i.astype(np.int64), j.astype(np.int64)
        assert (O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B) == p).all()
        keys = i * n + j
        assert len(np.unique(keys)) == len(keys)
        diag = i == j
        assert (w[diag] == support[i[diag]]).all()
        # present entries, by the definition
        for q in rng.choice(np.flatnonzero(~diag), 25, replace=False):
            assert w[q] == O.entry(inv, inv, int(i[q]), int(j[q])), (p, i[q], j[q])
        # absent pairs of this partition are zero by the definition
        present = set(keys.tolist())
        absent = 0
        while absent < 10:
            a, b = rng.integers(0, n, 2)
            if O.partition_of(np.array([a]), np.array([b]), P, ci.SEED_A, ci.SEED_B)[0] != p:
                continue
            if int(a) * n + int(b) in present:
                continue
            assert O.entry(inv, inv, int(a), int(b)) == 0.0
            absent += 1


def test_top_pairs(full):
    crp, T, L, plan, inv = full
    ti, tj, tw, _ = plan.topk(1000, upper=True)
    assert len(ti) == 1000 and (ti < tj).all()
    assert (np.diff(tw) <= 0).all()
    for q in range(20):
        assert tw[q] == O.entry(inv, inv, int(ti[q]), int(tj[q]))
    # no entry of a sampled partition above the 1000th weight is missing
    top = set((ti.astype(np.int64) * T.n_minor + tj).tolist())
    rng = np.random.default_rng(7)
    for p in rng.choice(P, 8, replace=False).tolist():
        i, j, w, _ = plan.export(p, p + 1)
        up = (i < j) & (w > tw[-1])
        for a, b in zip(i[up].tolist(), j[up].tolist()):
            assert a * T.n_minor + b in top


def test_whole_partitions_equal_the_oracle(full):
    """Two partitions, every entry: the oracle's partition_entries (the terms
    whose side hashes put them in partition p, summed) against the export,
    bit for bit -- offsetting errors inside a partition would show here."""
    crp, T, L, plan, inv = full
    Tc = O.Compressed.of(T)
    for p in (0, 517):
        want = O.partition_entries(Tc, Tc, P, p, ci.SEED_A, ci.SEED_B)
        i, j, w, _ = plan.export(p, p + 1)
        o = np.lexsort((j, i))
        assert np.array_equal(i[o].astype(np.int64), want.i)
        assert np.array_equal(j[o].astype(np.int64), want.j)
        assert np.array_equal(w[o], want.w)


def test_top1000_equals_the_oracle_certified_list(full):
    """The returned top 1000 (pairs i < j) equal, in order, the oracle's
    certified heaviest pairs of this very input (tests/golden/c2_top2000.txt,
    written by tests/golden/make_topk_fixtures.py; the fixture records the
    input's SHA-256)."""
    import hashlib
    import os
    crp, T, L, plan, inv = full
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_top2000.txt")
    rows, digest = [], None
    for line in open(path):
        if line.startswith("# input sha256 "):
            digest = line.split()[-1]
        elif line.strip() and not line.startswith("#"):
            rows.append(tuple(int(x) for x in line.split()))
    h = hashlib.sha256()
    h.update(T.ptr.tobytes())
    h.update(T.idx.tobytes())
    assert h.hexdigest() == digest, "the generator made a different input"
    ti, tj, tw, _ = plan.topk(1000, upper=True)
    got = list(zip(ti.tolist(), tj.tolist(), [int(x) for x in tw]))
    assert got == rows[:1000]
