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
    # the configuration bench.py times: 64 outer products per work item and
    # per-problem hot blocks of 128 items
    batch = crp.Batch([(x, x) for x in dev], Pb, ci.SEED_A, ci.SEED_B, tile_vectors=64,
                      hot_items=128)
    batch.run()
    _, terms = batch.sync()
    per = [int((T.lengths().astype(np.int64) ** 2).sum()) for T in Ts]
    assert terms == sum(per)
    rng = np.random.default_rng(5)
    # 64 of the problems under 1e6 terms, every entry against the oracle
    small = [q for q in range(len(Ts)) if per[q] < 1_000_000]
    for q in rng.choice(small, 64, replace=False).tolist():
        Tc = O.Compressed.of(Ts[q])
        ref = O.exact_product(Tc, Tc, O.FULL)
        i, j, w = batch.export(q)
        o = np.lexsort((j, i))
        assert np.array_equal(i[o], ref.i) and np.array_equal(j[o], ref.j), q
        assert np.array_equal(w[o], ref.w), q
    # 12 larger ones: every term stored once, the diagonal, sampled entries
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
    # top-1000 weight error, judged by the oracle's certified heaviest pairs of
    # this input: plain summary, and with 2^16 reserved counters chosen by the
    # network (trained on oracle counts of a separate stream of the recipe)
    # and by the product of marginals
    rows = _oracle_top_pairs("c4", T)
    n = T.n_minor
    m_pre = T.n_major // 100
    pre = crp.to_device(ci.Sparse(T.ptr[:m_pre + 1], T.idx[:T.ptr[m_pre]], None, n))
    params = _train_on_oracle_counts(crp, ci.C4)
    errs = {}
    for name, prm, reserve in (("plain", None, False), ("marginals", None, True),
                               ("predictor", params, True)):
        pl = crp.Plan(n, n, Ps, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER, summary_counters=ell,
                      reserved_counters=(1 << 16) if reserve else 0,
                      flags=crp.CRP_PLAN_SORTED_ROWS)
        if reserve:
            crp.predict_reserve(pl, pre, n, prm, 2048, 1 << 16)
        pl.accumulate(d, d)
        pl.sync()
        ti, tj, _, _ = pl.topk(1000, upper=True)
        errs[name] = _weight_error(ti, tj, rows, 1000)
        pl.close()
    print("c4 top-1000 weight error (oracle-judged):", errs)
    assert errs["predictor"][0] <= errs["plain"][0] + 1e-12
    assert errs["predictor"][1] == 0 and errs["plain"][1] == 0   # every pair weighed


def _oracle_top_pairs(name, T):
    """The oracle's certified heaviest pairs of this input from the fixture
    written by tests/golden/make_topk_fixtures.py (checked against the input's
    SHA-256)."""
    import glob
    import hashlib
    import os
    path = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden",
                                         f"{name}_top*.txt")))[0]
    rows, digest = [], None
    for line in open(path):
        if line.startswith("# input sha256 "):
            digest = line.split()[-1]
        elif line.strip() and not line.startswith("#"):
            a, b, c = line.split()
            rows.append((int(a), int(b), float(c)))
    h = hashlib.sha256()
    h.update(T.ptr.tobytes())
    h.update(T.idx.tobytes())
    assert h.hexdigest() == digest, "the generator made a different input"
    return rows


def _weight_error(ti, tj, rows, k):
    """1 - (true weight of the returned pairs) / (true top-k weight), and how
    many returned pairs lie outside the oracle's list (weight unknown)."""
    look = {(a, b): c for a, b, c in rows}
    got = [look.get((int(a), int(b))) for a, b in zip(ti, tj)]
    known = sum(x for x in got if x is not None)
    return 1.0 - known / sum(c for _, _, c in rows[:k]), sum(x is None for x in got)


def _train_on_oracle_counts(crp, w, m_train=200_000, R=2048):
    """The heavy-pair network trained on a separate stream of the recipe:
    features of the candidate pairs from its 1% prefix, labels log(1 + count)
    from the oracle's exact product of that stream."""
    import torch
    tr = ci.transactions(w.seed + 17, m_train, w.n, w.lam, w.lmin, w.lmax, w.zipf_s)
    ref = O.exact_product(O.Compressed.of(tr), O.Compressed.of(tr), O.UPPER)
    keys = ref.i * w.n + ref.j
    m_tp = m_train // 100
    cpre = crp.to_device(ci.Sparse(tr.ptr[:m_tp + 1], tr.idx[:tr.ptr[m_tp]], None, w.n))
    cI, cJ, X = crp.candidate_pairs(cpre, w.n, R)
    ck = cI.cpu().numpy().astype(np.int64) * w.n + cJ.cpu().numpy()
    pos = np.minimum(np.searchsorted(keys, ck), len(keys) - 1)
    y = np.log1p(np.where(keys[pos] == ck, ref.w[pos], 0.0))
    Y = torch.tensor(y / max(y.max(), 1e-9), dtype=torch.float32, device="cuda")
    params = crp.mlp_init(7)
    trainer = crp.MLPTrainer(params, lr=3e-3)
    losses = [trainer.step(X, Y) for _ in range(300)]
    assert losses[-1] < losses[0]
    return params
