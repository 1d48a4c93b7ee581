"""Pins of the oracle's Count-Sketch (Preliminaries; Figure 1) against what
the mathematics fixes: exhaustive pairwise independence of the sign hash at
small word widths, the dense matrix product (numpy), the per-term loop of
Figure 1, the exact estimate of an entry alone in its partition, and the
unbiasedness and variance of the estimator over many seeds."""
import itertools

import numpy as np
import pytest

from oracle import crp_oracle as O


def _rand_sparse(rng, K, n, density, integer=True):
    ptr = [0]
    idx = []
    for _ in range(K):
        L = rng.binomial(n, density)
        idx.extend(np.sort(rng.choice(n, size=L, replace=False)).tolist())
        ptr.append(len(idx))
    if integer:
        val = rng.integers(1, 4, size=len(idx)).astype(np.float32)
    else:
        val = rng.uniform(0.1, 2.0, size=len(idx)).astype(np.float32)
    return O.Compressed(np.array(ptr, np.int64), np.array(idx, np.int32), val, n)


# ---------------------------------------------------------------------------
# The sign hash
# ---------------------------------------------------------------------------

def test_side_sign_is_the_top_bit_of_multiply_add():
    # s(x) = 1 - 2 * (one-bit multiply-add-shift), the construction whose
    # pairwise independence is checked exhaustively at small widths.
    rng = np.random.default_rng(5)
    for seed in (0, 1, 0x243F6A8885A308D3):
        c, d = O.sign_params(seed)
        assert (c, d) == tuple(O.splitmix64(seed, 4)[2:4])
        xs = rng.integers(0, 2**31, 50)
        want = [1 - 2 * O.mas_hash_scalar(int(x), c, d, 1) for x in xs]
        assert O.side_sign(xs, seed).tolist() == want


def test_pair_sign_is_pairwise_independent_exhaustively():
    # s(i, j) = s_a(i) s_b(j) with one-bit multiply-add-shift on 6-bit words
    # and 3-bit keys: over all (c_a, d_a, c_b, d_b), for every two distinct
    # pairs the two signs are equal exactly half the time, and each sign is
    # +1 exactly half the time.
    w = 6
    c, d = np.meshgrid(np.arange(1 << w), np.arange(1 << w), indexing="ij")
    c, d = c.ravel(), d.ravel()

    def s(x):
        return 1 - 2 * ((((c * x) + d) & ((1 << w) - 1)) >> (w - 1))

    side = {x: s(x) for x in range(8)}
    n = len(c)
    for x in range(8):
        assert (side[x] == 1).sum() * 2 == n
    pairs = list(itertools.product(range(8), range(8)))
    for (i, j), (k, l) in itertools.combinations(pairs, 2):
        pa = side[i] * side[k]          # product over the a-side draws
        pb = side[j] * side[l]          # product over the b-side draws
        # Pr[s(i,j) s(k,l) = +1] over independent a and b draws
        plus = (pa == 1).sum() * (pb == 1).sum() + (pa == -1).sum() * (pb == -1).sum()
        assert plus * 2 == n * n, ((i, j), (k, l))


def test_pair_signs_are_uncorrelated_over_seeds():
    # Over independent side seeds, the signs of the diagonal entry, of an
    # entry and its transpose, and of two entries sharing a row are each
    # +/-1 with mean 0 -- a sign drawn from one side only, or shared by the
    # two sides, fails one of them.
    R = 4000
    seeds = range(R)
    diag = np.array([O.sign_of(np.array([5]), np.array([5]), 2 * r + 1, 2 * r + 2)[0] for r in seeds])
    tr = np.array([O.sign_of(np.array([3, 9]), np.array([9, 3]), 2 * r + 1, 2 * r + 2).prod() for r in seeds])
    row = np.array([O.sign_of(np.array([4, 4]), np.array([1, 8]), 2 * r + 1, 2 * r + 2).prod() for r in seeds])
    col = np.array([O.sign_of(np.array([1, 8]), np.array([4, 4]), 2 * r + 1, 2 * r + 2).prod() for r in seeds])
    bound = 4.0 / np.sqrt(R)
    for v in (diag, tr, row, col):
        assert set(np.unique(v).tolist()) == {-1, 1}
        assert abs(v.mean()) < bound


# ---------------------------------------------------------------------------
# The sketch
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [O.FULL, O.UPPER])
@pytest.mark.parametrize("P", [1, 4, 32])
def test_count_sketch_matches_dense_product(mode, P):
    # CS[p] = sum over entries in partition p of w s, with the entries taken
    # from the dense product A^T B (numpy) instead of the outer products.
    rng = np.random.default_rng(100 + P + mode)
    A = _rand_sparse(rng, 30, 25, 0.2)
    B = _rand_sparse(rng, 30, 20, 0.2)
    C = O.dense(A).T @ O.dense(B)
    i, j = np.nonzero(C)
    if mode == O.UPPER:
        keep = i < j
        i, j = i[keep], j[keep]
    w = C[i, j]
    want = np.zeros(P)
    p = O.partition_of(i, j, P, 11, 22)
    s = O.sign_of(i, j, 11, 22)
    for q in range(len(i)):
        want[p[q]] += w[q] * s[q]
    got = O.count_sketch(O.exact_product(A, B, mode), P, 11, 22)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", [O.FULL, O.UPPER])
def test_count_sketch_per_term_equals_per_entry(mode):
    # Figure 1 adds every term; summing the terms of an entry first gives the
    # same sketch exactly on integer weights.
    rng = np.random.default_rng(7 + mode)
    A = _rand_sparse(rng, 40, 30, 0.15)
    B = _rand_sparse(rng, 40, 30, 0.15)
    for P in (1, 8, 64):
        a = O.count_sketch_terms(A, B, P, 3, 4, mode)
        b = O.count_sketch(O.exact_product(A, B, mode), P, 3, 4)
        assert np.array_equal(a, b)


def test_isolated_entry_is_estimated_exactly():
    # A single nonzero entry: its partition holds nothing else, so the
    # estimate is its weight for every seed and partition count, and every
    # other partition of the sketch is zero.
    ptr = np.array([0, 1], np.int64)
    A = O.Compressed(ptr, np.array([3], np.int32), np.array([2.0], np.float32), 10)
    B = O.Compressed(ptr, np.array([7], np.int32), np.array([3.5], np.float32), 10)
    prod = O.exact_product(A, B)
    for seed_a, seed_b in ((1, 2), (5, 9), (0x243F6A8885A308D3, 0x13198A2E03707344)):
        for P in (1, 16, 1024):
            cs = O.count_sketch(prod, P, seed_a, seed_b)
            assert O.sketch_estimate(cs, np.array([3]), np.array([7]), P, seed_a, seed_b)[0] == 7.0
            assert np.count_nonzero(cs) == 1
            assert abs(cs).sum() == 7.0


def test_estimate_is_unbiased_with_the_collision_variance():
    # Over independent seeds, estimate - w_e = sum over other entries e' in
    # h(e)'s partition of w_e' s(e) s(e'): mean 0, variance
    # sum_{e' != e} w_e'^2 Pr[h(e') = h(e)] = sum w_e'^2 / P.
    rng = np.random.default_rng(31)
    A = _rand_sparse(rng, 50, 40, 0.2)
    B = _rand_sparse(rng, 50, 40, 0.2)
    prod = O.exact_product(A, B)
    P = 16
    q = int(np.argmax(prod.w))
    ei, ej, ew = prod.i[q:q + 1], prod.j[q:q + 1], prod.w[q]
    var = (np.sum(prod.w ** 2) - ew ** 2) / P
    R = 600
    err = np.empty(R)
    for r in range(R):
        sa, sb = 1000 + 2 * r, 1001 + 2 * r
        cs = O.count_sketch(prod, P, sa, sb)
        err[r] = O.sketch_estimate(cs, ei, ej, P, sa, sb)[0] - ew
    assert abs(err.mean()) < 4.0 * np.sqrt(var / R)
    assert 0.6 * var < np.mean(err ** 2) < 1.5 * var


def test_median_of_instances_beats_one_instance():
    # The median of t independent estimates concentrates: on a skewed matrix
    # the median error of the heaviest entries over t = 11 instances is below
    # the mean absolute error of a single instance.
    rng = np.random.default_rng(77)
    A = _rand_sparse(rng, 200, 60, 0.08)
    B = _rand_sparse(rng, 200, 60, 0.08)
    prod = O.exact_product(A, B)
    P = 64
    top = np.argsort(-prod.w, kind="stable")[:20]
    ests = []
    for t in range(11):
        sa, sb = 500 + 2 * t, 501 + 2 * t
        cs = O.count_sketch(prod, P, sa, sb)
        ests.append(O.sketch_estimate(cs, prod.i[top], prod.j[top], P, sa, sb))
    ests = np.array(ests)
    med = O.sketch_median(ests)
    assert np.array_equal(med, np.sort(ests, axis=0)[5])
    one = np.abs(ests - prod.w[top]).mean()
    assert np.abs(med - prod.w[top]).mean() < one


@pytest.mark.parametrize("P", [1, 8, 64])
@pytest.mark.parametrize("values", [False, True])
def test_sketch_spectrum_is_the_fft_of_the_sketch(P, values):
    # The closed form computed from the inputs alone equals the discrete
    # Fourier transform (numpy FFT) of the sketch built from the entries;
    # empty vectors at the start, middle and end take part.
    rng = np.random.default_rng(60 + P + values)
    A = _rand_sparse(rng, 45, 30, 0.2, integer=not values)
    B = _rand_sparse(rng, 45, 25, 0.2, integer=not values)
    A = _with_empty(A, (0, 10, 11, 44))   # empty vectors: first, a middle run, last
    B = _with_empty(B, (0, 10, 11, 44))
    cs = O.count_sketch(O.exact_product(A, B), P, 13, 17)
    freqs = list(range(P))
    got = O.count_sketch_spectrum(A, B, P, 13, 17, freqs)
    want = np.conj(np.fft.fft(cs)) if P > 1 else np.array([cs.sum()], dtype=complex)
    # sum_p CS[p] exp(+2 pi i f p / P) is the conjugate of numpy's forward FFT
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)


def _with_empty(X, ks):
    ptr, idx = [0], []
    val = [] if X.val is not None else None
    for k in range(X.n_major):
        s, e = int(X.ptr[k]), int(X.ptr[k + 1])
        if k not in ks:
            idx.extend(X.idx[s:e].tolist())
            if val is not None:
                val.extend(X.val[s:e].tolist())
        ptr.append(len(idx))
    return O.Compressed(np.array(ptr, np.int64), np.array(idx, np.int32),
                        None if val is None else np.array(val, np.float32), X.n_minor)
