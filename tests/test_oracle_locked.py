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
