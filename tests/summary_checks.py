"""Checks of per-partition Space-Saving buckets that hold for the sequential
algorithm of the Preliminaries on any arrival order of each partition's
terms (shared by the GPU tests and the oracle's own check)."""
import numpy as np

import crp_inputs as ci
from oracle import crp_oracle as O


def _truth(A, B, P, mode=O.FULL):
    ref = O.exact_product(A, B, mode)
    part = O.partition_of(ref.i, ref.j, P, ci.SEED_A, ci.SEED_B)
    true = dict(zip((ref.i.astype(np.int64) * B.n_minor + ref.j).tolist(), ref.w.tolist()))
    W = np.bincount(part, weights=ref.w, minlength=P)
    distinct = np.bincount(part, minlength=P)
    return ref, part, true, W, distinct


def _check_buckets(i, j, up, lo, P, ell, n_cols, true, W, distinct, ref, part):
    p = O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B)
    keys = i.astype(np.int64) * n_cols + j
    assert len(np.unique(keys)) == len(keys)
    n_keys = np.bincount(p, minlength=P)
    assert (n_keys <= ell).all()
    # counts of a bucket add up to its partition's weight, exactly
    assert np.array_equal(np.bincount(p, weights=up, minlength=P), W)
    tv = np.array([true.get(int(k), 0.0) for k in keys])
    assert (lo <= tv).all() and (tv <= up).all()
    err = up - lo
    mins = np.full(P, np.inf)
    np.minimum.at(mins, p, up)
    full = n_keys == ell
    assert (err[full[p]] <= mins[p][full[p]]).all()
    assert (err == 0)[~full[p]].all()     # a bucket never filled never replaced
    assert (mins[full] <= W[full] / ell).all()
    # heavy keys are recorded; partitions with <= ell distinct keys are exact
    present = set(keys.tolist())
    heavy = ref.w > W[part] / ell
    for a, b in zip(ref.i[heavy].tolist(), ref.j[heavy].tolist()):
        assert a * n_cols + b in present
    small = distinct <= ell
    assert (n_keys[small] == distinct[small]).all()
    assert (err[small[p]] == 0).all()
    assert np.array_equal(up[small[p]], tv[small[p]])
