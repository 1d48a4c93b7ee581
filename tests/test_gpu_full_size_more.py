"""Parity at the full sizes of the real-valued Markov expansion (C = A A,
100,000 x 100,000), the batched workload (4,096 problems in one launch) and
the heavy-entry summaries (50,000,000 transactions x 1,000,000 items), in the
configurations bench.py times: properties that hold at any size, and sampled
entries computed one by one by the oracle from the definition of an entry as
an inner product.  (A module of its own, so that the 10M-transaction plan of
the co-occurrence test has released its device memory first.)"""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O

pytestmark = pytest.mark.gpu


# ---------------------------------------------------------------------------
# The real-valued Markov expansion C = A A at full size (100,000 x 100,000)
# ---------------------------------------------------------------------------

def test_markov_expansion_full_size():
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp
    A, At = ci.c3()                      # CSC of A (a_k = column k), CSR of A (b_k = row k)
    n = A.n_minor
    Pm = 1024
    plan = crp.Plan(n, n, Pm, ci.SEED_A, ci.SEED_B, value_type=crp.CRP_F32_COMP, groups=0,
                    flags=crp.CRP_PLAN_ROUTED, auto_grow=True)
    plan.accumulate(crp.to_device(A), crp.to_device(At))
    plan.sync()
    st = plan.stats()
    assert st["terms"] == int((A.lengths().astype(np.int64) * At.lengths().astype(np.int64)).sum())
    rows, cols = O.Compressed.of(At), O.Compressed.of(A)   # rows of A, columns of A
    rng = np.random.default_rng(11)
    for p in rng.choice(Pm, 3, replace=False).tolist():
        i, j, w, _ = plan.export(p, p + 1)
        assert (O.partition_of(i, j, Pm, ci.SEED_A, ci.SEED_B) == p).all()
        for q in rng.choice(len(i), 20, replace=False):
            want = O.entry(rows, cols, int(i[q]), int(j[q]))
            assert abs(w[q] - want) <= 1e-6 * abs(want), (i[q], j[q], w[q], want)
    ti, tj, tw, _ = plan.topk(50)
    for a, b, v in zip(ti.tolist(), tj.tolist(), tw.tolist()):
        want = O.entry(rows, cols, a, b)
        assert abs(v - want) <= 1e-6 * abs(want)
    plan.close()


# ---------------------------------------------------------------------------
# The batched workload at full size: 4,096 problems in one launch
# ---------------------------------------------------------------------------

def test_batched_full_size():
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp
    ws = ci.c5_params()
    Ts = [w.generate() for w in ws]
    dev = [crp.to_device(T) for T in Ts]
    Pb = 256
    batch = crp.Batch([(x, x) for x in dev], Pb, ci.SEED_A, ci.SEED_B, tile_vectors=32)
    batch.run()
    _, terms = batch.sync()
    per = [int((T.lengths().astype(np.int64) ** 2).sum()) for T in Ts]
    assert terms == sum(per)
    rng = np.random.default_rng(5)
    for q in rng.choice(len(Ts), 12, replace=False).tolist():
        T = Ts[q]
        i, j, w = batch.export(q)
        assert int(w.astype(np.int64).sum()) == per[q]          # every term stored once
        keys = i.astype(np.int64) * T.n_minor + j
        assert len(np.unique(keys)) == len(keys)
        inv = O.Compressed.of(ci.transpose(T))
        support = np.diff(inv.ptr)
        diag = i == j
        assert (w[diag] == support[i[diag]]).all()
        for x in rng.choice(len(i), min(10, len(i)), replace=False):
            assert w[x] == O.entry(inv, inv, int(i[x]), int(j[x]))
    batch.close()


# ---------------------------------------------------------------------------
# The heavy-entry summaries at full size (50,000,000 transactions x 1,000,000
# items, pairs i < j, 2^20 counters per partition)
# ---------------------------------------------------------------------------

def test_heavy_entry_summaries_full_size():
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp
    T = ci.C4.generate()
    Ps, ell = 256, 1 << 20
    plan = crp.Plan(T.n_minor, T.n_minor, Ps, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER,
                    summary_counters=ell, flags=crp.CRP_PLAN_SORTED_ROWS)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    L = T.lengths().astype(np.int64)
    assert plan.stats()["terms"] == int((L * (L - 1) // 2).sum())
    inv = O.Compressed.of(ci.transpose(T))
    rng = np.random.default_rng(3)
    for p in rng.choice(Ps, 2, replace=False).tolist():
        i, j, up, lo = plan.export(p, p + 1)
        assert 0 < len(i) <= ell and (i < j).all()
        assert (O.partition_of(i, j, Ps, ci.SEED_A, ci.SEED_B) == p).all()
        for x in rng.choice(len(i), 20, replace=False):
            t = O.entry(inv, inv, int(i[x]), int(j[x]))
            assert lo[x] <= t <= up[x], (i[x], j[x], lo[x], t, up[x])
    ti, tj, tu, tl = plan.topk(1000, upper=True)
    for a, b, u, l in list(zip(ti.tolist(), tj.tolist(), tu.tolist(), tl.tolist()))[:20]:
        t = O.entry(inv, inv, a, b)
        assert l <= t <= u
    plan.close()
