"""Batched products: many independent co-occurrence problems of uneven size in
one persistent, graph-captured launch, each problem bit-exact against the
oracle; bounded waits on withheld inputs report CRP_ETIMEOUT (no GPU hang)."""
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


@pytest.fixture(scope="module")
def problems():
    # the batched workload's recipe (log-uniform sizes, Zipf s in [0.8, 1.3],
    # Poisson(12) lengths) at sizes the oracle finishes quickly
    ws = ci.c5_params(40, m_range=(100, 4000), n_range=(100, 3000))
    return [w.generate() for w in ws]


def _exact(T, mode):
    Tc = O.Compressed.of(T)
    return O.exact_product(Tc, Tc, mode)


def _check(batch, q, ref):
    i, j, w = batch.export(q)
    o = np.lexsort((j, i))
    assert np.array_equal(i[o], ref.i) and np.array_equal(j[o], ref.j), q
    assert np.array_equal(w[o], ref.w), q


@pytest.mark.parametrize("mode", [O.FULL, O.UPPER])
def test_batch_each_problem_bit_exact(crp, problems, mode):
    dev = [crp.to_device(T) for T in problems]
    batch = crp.Batch([(d, d) for d in dev], 64, ci.SEED_A, ci.SEED_B, mode=mode, tile_vectors=16)
    refs = [_exact(T, mode) for T in problems]
    for rep in range(2):          # the captured graph resets and refills the tables
        batch.run()
        ms, terms = batch.sync()
        assert terms == sum(r.terms for r in refs)
        for q, ref in enumerate(refs):
            _check(batch, q, ref)
    info = batch.info()
    assert info["total_terms"] == sum(int((T.lengths().astype(np.int64) ** 2).sum())
                                      for T in problems)
    batch.close()


def test_batch_matches_one_plan_per_problem(crp, problems):
    dev = [crp.to_device(T) for T in problems[:12]]
    batch = crp.Batch([(d, d) for d in dev], 256, ci.SEED_A, ci.SEED_B)
    batch.run()
    batch.sync()
    for q, (T, d) in enumerate(zip(problems[:12], dev)):
        plan = crp.Plan(T.n_minor, T.n_minor, 256, ci.SEED_A, ci.SEED_B,
                        flags=crp.CRP_PLAN_DIRECT)
        plan.accumulate(d, d)
        plan.sync()
        a = plan.export()
        b = batch.export(q)
        oa, ob = np.lexsort((a[1], a[0])), np.lexsort((b[1], b[0]))
        for x, y in zip(a[:3], b):
            assert np.array_equal(x[oa], y[ob])
        plan.close()
    batch.close()


def test_withheld_problem_times_out_then_completes(crp, problems):
    dev = [crp.to_device(T) for T in problems[:10]]
    batch = crp.Batch([(d, d) for d in dev], 64, ci.SEED_A, ci.SEED_B,
                      wait_timeout_ns=200_000_000)
    batch.set_ready(3, False)
    batch.run()
    with pytest.raises(crp.CrpError) as e:
        batch.sync()
    assert e.value.status == crp.CRP_ETIMEOUT
    for q in (0, 1, 2, 4, 9):          # the others finished exactly
        _check(batch, q, _exact(problems[q], O.FULL))
    i, j, w = batch.export(3)
    assert len(i) == 0                 # the withheld problem was skipped
    batch.set_ready(3, True)           # the context is still usable
    batch.run()
    batch.sync()
    _check(batch, 3, _exact(problems[3], O.FULL))
    batch.close()


def test_batch_autotuned_choice_is_bit_exact(crp, problems, tmp_path):
    """crp_autotune_batch picks P, tile_vectors and the per-problem hot block on
    a sample of the problems;
    the batch built with its choice is bit-exact on every problem, and a
    second call with the same cache file returns the cached choice."""
    dev = [crp.to_device(T) for T in problems]
    pairs = [(d, d) for d in dev]
    cache = str(tmp_path / "tune.txt")
    kw, tps = crp.autotune_batch(pairs, ci.SEED_A, ci.SEED_B, sample_probs=16, cache_path=cache)
    assert kw["P"] in (64, 256, 1024, 4096) and kw["tile_vectors"] in (16, 32, 64, 128)
    assert kw["hot_items"] in (0, 64, 128, 255)
    assert tps > 0
    kw2, tps2 = crp.autotune_batch(pairs, ci.SEED_A, ci.SEED_B, sample_probs=16, cache_path=cache)
    assert kw2 == kw and tps2 == tps
    batch = crp.Batch(pairs, kw["P"], ci.SEED_A, ci.SEED_B, tile_vectors=kw["tile_vectors"],
                      hot_items=kw["hot_items"])
    batch.run()
    batch.sync()
    for q, T in enumerate(problems):
        _check(batch, q, _exact(T, O.FULL))
    batch.close()


@pytest.mark.parametrize("mode,R", [(O.FULL, 64), (O.UPPER, 64), (O.FULL, 255), (O.FULL, 7)])
def test_batch_hot_tier_bit_exact(crp, problems, mode, R):
    """Per-problem dense tier: pairs of two of a problem's R most frequent
    items (on its first outer products) count in the problem's hot block and
    are added into its tables after the persistent kernel; every problem stays
    bit-exact, run after run (the graph recounts, reselects and clears)."""
    dev = [crp.to_device(T) for T in problems]
    batch = crp.Batch([(d, d) for d in dev], 64, ci.SEED_A, ci.SEED_B, mode=mode, tile_vectors=16,
                      hot_items=R)
    refs = [_exact(T, mode) for T in problems]
    for rep in range(2):
        batch.run()
        ms, terms = batch.sync()
        assert terms == sum(r.terms for r in refs)
        for q, ref in enumerate(refs):
            _check(batch, q, ref)
    batch.close()


def test_batch_hot_tier_two_sides(crp, problems):
    """A and B different arrays (same number of outer products): each side
    selects its own hot items; every problem bit-exact against the oracle's
    A^T B."""
    import dataclasses
    ws = ci.c5_params(40, m_range=(100, 4000), n_range=(100, 3000))[:12]
    others = [dataclasses.replace(w, seed=w.seed + 7).generate() for w in ws]
    pairs, refs = [], []
    for T, U in zip(problems[:12], others):
        assert T.n_major == U.n_major
        pairs.append((crp.to_device(T), crp.to_device(U)))
        refs.append(O.exact_product(O.Compressed.of(T), O.Compressed.of(U), O.FULL))
    batch = crp.Batch(pairs, 64, ci.SEED_A, ci.SEED_B, tile_vectors=16, hot_items=32)
    batch.run()
    batch.sync()
    for q, ref in enumerate(refs):
        _check(batch, q, ref)
    batch.close()
