"""The launch-configuration autotuner: its choice is a valid plan whose result
is bit-exact, and a cached entry is reused."""
import os

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


def test_autotune_choice_is_exact_and_cached(crp, tmp_path):
    T = ci.C2.scaled(m=40_000, n=5_000).generate()
    d = crp.to_device(T)
    cache = str(tmp_path / "tune.txt")
    kw, tps = crp.autotune(d, d, T.n_minor, T.n_minor, ci.SEED_A, ci.SEED_B,
                           sample_vectors=20_000, cache_path=cache)
    assert tps > 0 and kw["P"] in (256, 1024, 4096)
    assert os.path.exists(cache) and len(open(cache).read().splitlines()) == 1
    kw2, tps2 = crp.autotune(d, d, T.n_minor, T.n_minor, ci.SEED_A, ci.SEED_B,
                             sample_vectors=20_000, cache_path=cache)
    assert kw2 == kw and abs(tps2 - tps) <= 1e-6 * tps     # served from the cache
    assert len(open(cache).read().splitlines()) == 1
    plan = crp.Plan(T.n_minor, T.n_minor, seed_a=ci.SEED_A, seed_b=ci.SEED_B, **kw)
    plan.accumulate(d, d)
    plan.sync()
    i, j, w, _ = plan.export()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    o = np.lexsort((j, i))
    assert np.array_equal(i[o], ref.i) and np.array_equal(j[o], ref.j)
    assert np.array_equal(w[o], ref.w)
    plan.close()


def test_plan_with_P_zero_tunes_at_its_first_call(crp):
    # P = 0: the first accumulate tunes the plan on its first outer products and
    # the plan becomes the chosen one; later calls add to it
    T = ci.C2.scaled(m=30_000, n=3_000).generate()
    Tc = O.Compressed.of(T)
    half = T.n_major // 2
    parts = [ci.Sparse(T.ptr[lo:hi + 1] - T.ptr[lo], T.idx[T.ptr[lo]:T.ptr[hi]], None, T.n_minor)
             for lo, hi in ((0, half), (half, T.n_major))]
    plan = crp.Plan(T.n_minor, T.n_minor, 0, ci.SEED_A, ci.SEED_B, auto_grow=True)
    assert plan.partition_of(5, 7) == 0 and len(plan.topk(10)[0]) == 0   # placeholder
    for part in parts:
        dd = crp.to_device(part)
        plan.accumulate(dd, dd)
    plan.sync()
    assert plan.P in (256, 1024, 4096)
    ref = O.exact_product(Tc, Tc, O.FULL)
    i, j, w, _ = plan.export()
    o = np.lexsort((j, i))
    assert np.array_equal(i[o], ref.i) and np.array_equal(j[o], ref.j)
    assert np.array_equal(w[o], ref.w)
    assert plan.partition_of(5, 7) == int(O.partition_of(np.array([5]), np.array([7]), plan.P,
                                                          ci.SEED_A, ci.SEED_B)[0])
    with pytest.raises(crp.CrpError):
        crp.Plan(100, 100, 0, 1, 2, summary_counters=4)
    plan.close()
