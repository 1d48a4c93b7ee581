"""The bucket checks used on the GPU's locked summaries, run on the oracle's
sequential Space-Saving (Preliminaries) over the canonical order of each
partition's terms: one of the summaries a lock may produce passes them, so the
checks demand nothing the sequential algorithm does not give."""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O
from summary_checks import _check_buckets, _truth


@pytest.mark.parametrize("P,ell", [(64, 2), (16, 1), (8, 5)])
def test_oracle_sequential_space_saving_has_the_bucket_invariants(P, ell):
    # the oracle's sequential Space-Saving on the canonical order of each
    # partition's terms is one of the summaries the lock may produce: the
    # same checks pass on it
    T = ci.C1.scaled(m=5000).generate()
    Tc = O.Compressed.of(T)
    ref, part, true, W, distinct = _truth(Tc, Tc, P)
    streams = O.partition_streams(Tc, Tc, P, ci.SEED_A, ci.SEED_B)
    I, J, U, L = [], [], [], []
    for p in range(P):
        ss = O.space_saving(streams[p], ell)
        for key, (c, e) in ss.items():
            a, b = divmod(key, 1000)
            I.append(a)
            J.append(b)
            U.append(c)
            L.append(c - e)
    _check_buckets(np.array(I), np.array(J), np.array(U, float), np.array(L, float), P, ell, 1000,
                   true, W, distinct, ref, part)


@pytest.mark.parametrize("P,ell,mode", [(16, 2, O.FULL), (64, 3, O.UPPER), (1, 4, O.FULL)])
def test_bucket_summaries_equal_the_per_partition_streams(P, ell, mode):
    # the grouped form returns, bucket by bucket, what Space-Saving gives on
    # each partition's stream taken one partition at a time
    T = ci.C1.scaled(m=3000).generate()
    Tc = O.Compressed.of(T)
    p, key, cnt, over = O.bucket_summaries(Tc, Tc, P, ell, ci.SEED_A, ci.SEED_B, mode)
    streams = O.partition_streams(Tc, Tc, P, ci.SEED_A, ci.SEED_B, mode)
    want = {}
    for q in range(P):
        for k, (c, o) in O.space_saving(streams[q], ell).items():
            want[(q, k)] = (c, o)
    got = {(int(a), int(b)): (c, o) for a, b, c, o in zip(p, key, cnt, over)}
    assert got == want
    # every bucket's counts add up to its stream's weight
    W = np.zeros(P)
    for q in range(P):
        W[q] = sum(w for _, w in streams[q])
    assert np.array_equal(np.bincount(p, weights=cnt, minlength=P), W)
