"""The seeded input generators (shared by the CUDA path and the oracle)."""
import os

import numpy as np

import crp_inputs as ci

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        ctr, key, out = w[:4], w[4:6], w[6:]
        assert ci.philox_block(key[0] | (key[1] << 32), tuple(ctr)) == tuple(out)


def test_transactions_shape_and_determinism():
    T = ci.C1.generate()
    T2 = ci.C1.generate()
    assert np.array_equal(T.ptr, T2.ptr) and np.array_equal(T.idx, T2.idx)
    L = T.lengths()
    assert L.min() >= 2 and L.max() <= 40
    assert abs(L.mean() - 10) < 0.2
    for t in range(0, T.n_major, 997):
        row = T.idx[T.ptr[t]:T.ptr[t + 1]]
        assert (np.diff(row) > 0).all()           # sorted, distinct
        assert row.min() >= 0 and row.max() < 1000
    # Zipf(1.1): away from the saturated head (rank 1 sits in most
    # transactions), supports of ranks 50 and 100 are in ratio ~2^1.1
    sup = np.bincount(T.idx, minlength=1000)
    assert sup.argmax() == 0
    r = sup[45:55].sum() / sup[95:105].sum()
    assert 1.9 < r < 2.4, r


def test_unclamped_lengths_allow_empty_and_singleton_rows():
    T = ci.transactions(1, 20000, 5000, 1.5, 0, -1, 1.2)
    L = T.lengths()
    assert (L == 0).any() and (L == 1).any()


def test_stochastic_columns():
    A, At = ci.c3(n=5000, cmax=400)
    L = A.lengths()
    assert L.min() >= 5 and L.max() <= 400
    sums = np.add.reduceat(A.val.astype(np.float64), A.ptr[:-1])
    assert np.abs(sums - 1).max() < 1e-5
    assert (A.val > 0).all()
    # the transpose holds the same entries
    assert At.nnz == A.nnz
    D = np.zeros((5000, 5000), np.float32)
    for k in range(0, 5000, 250):
        D[A.idx[A.ptr[k]:A.ptr[k + 1]], k] = A.val[A.ptr[k]:A.ptr[k + 1]]
    for r in range(0, 5000, 777):
        cols = At.idx[At.ptr[r]:At.ptr[r + 1]]
        vals = At.val[At.ptr[r]:At.ptr[r + 1]]
        m = cols % 250 == 0
        assert np.array_equal(D[r, cols[m]], vals[m])


def test_c5_params_ranges():
    ps = ci.c5_params(64)
    assert all(100 <= p.m <= 200_000 and 1000 <= p.n <= 100_000 for p in ps)
    assert all(0.8 <= p.zipf_s <= 1.3 for p in ps)
    assert len({p.seed for p in ps}) == 64
