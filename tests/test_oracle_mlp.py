"""Pins of the oracle's predictor network: its backward pass against central
finite differences (rounding off, fp64), bf16 rounding against its definition,
and Adam on a quadratic."""
import numpy as np
import pytest

from oracle import crp_oracle as O


def test_bf16_round_definition():
    # representable values are fixed points; ties go to even; spacing at 1 is 2^-7
    for v in (1.0, -2.5, 0.0, 3.140625, 2.0 ** -20):
        assert O.bf16_round(v) == v
    assert O.bf16_round(1.0 + 2 ** -8) == 1.0            # tie -> even (1.0)
    assert O.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even
    assert O.bf16_round(1.0 + 2 ** -8 + 2 ** -12) == 1.0 + 2 ** -7
    x = np.random.default_rng(0).normal(size=1000)
    r = O.bf16_round(x)
    assert (np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_mlp_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    theta = O.mlp_init(seed)
    X = rng.uniform(0, 1, (37, 2))
    t = rng.uniform(0, 1, 37)
    L, g, _ = O.mlp_loss_grad(theta, X, t, rounding=False)
    idx = rng.choice(len(theta), 60, replace=False)
    h = 1e-6
    for q in idx:
        e = np.zeros_like(theta)
        e[q] = h
        Lp, _, _ = O.mlp_loss_grad(theta + e, X, t, rounding=False)
        Lm, _, _ = O.mlp_loss_grad(theta - e, X, t, rounding=False)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, g[q])


def test_mlp_forward_closed_form_single_unit():
    # one active hidden path: W1 row 0 = (1, 0), everything else zero
    d = {n: np.zeros(s) for n, s in O.MLP_SIZES}
    d["W1"][0, 0] = 1.0
    d["W2"][0, 0] = 2.0
    d["w3"][0] = 3.0
    d["b3"][0] = 0.5
    theta = O.mlp_pack(d)
    X = np.array([[0.25, 9.0], [-1.0, 4.0]])
    y, _ = O.mlp_forward(theta, X)
    assert np.allclose(y, [3 * 2 * 0.25 + 0.5, 0.5])


def test_adam_minimises_quadratic():
    theta = np.array([3.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for s in range(1, 2001):
        theta, m, v = O.adam_step(theta, m, v, 2 * theta, 0.05, s)
    assert np.abs(theta).max() < 1e-2


def test_marginal_features_closed_form():
    # log(1 + c) / log(1 + max c) at counts 0, 9, 99 with max 99:
    # log 1 = 0, log 10 / log 100 = 1/2, log 100 / log 100 = 1
    X = O.marginal_features(np.array([0, 9, 99]), np.array([99, 0, 9]), np.log(100.0))
    np.testing.assert_allclose(X, [[0.0, 1.0], [0.5, 0.0], [1.0, 0.5]], rtol=1e-15, atol=0)


def test_prefix_counts_and_candidate_pairs_against_dense_and_brute_force():
    rng = np.random.default_rng(3)
    m, n, R = 300, 40, 9
    ptr = [0]
    idx = []
    for _ in range(m):
        L = rng.integers(0, 8)
        # Zipf-like item draws so that counts differ and some tie
        sel = np.unique(np.minimum(rng.zipf(1.6, L) - 1, n - 1))
        idx.extend(sel.tolist())
        ptr.append(len(idx))
    T = O.Compressed(np.array(ptr, np.int64), np.array(idx, np.int32), None, n)
    c = O.prefix_item_counts(T)
    assert np.array_equal(c, O.dense(T).sum(axis=0).astype(np.int64))   # column sums
    top = O.top_items(c, R)
    brute = sorted(range(n), key=lambda x: (-c[x], x))[:R]
    assert top.tolist() == brute
    i, j, X, c2 = O.candidate_pairs(T, R)
    assert np.array_equal(c2, c)
    assert len(i) == R * (R - 1) // 2 and (i < j).all()
    assert set(i.tolist()) | set(j.tolist()) == set(brute)
    assert len(set(zip(i.tolist(), j.tolist()))) == len(i)
    mx = c.max()
    # the most frequent item's feature is 1; an item of count 0 would be 0
    for a, b, x in zip(i, j, X):
        if c[a] == mx:
            assert x[0] == 1.0
        if c[b] == mx:
            assert x[1] == 1.0
        assert 0.0 <= x[0] <= 1.0 and 0.0 <= x[1] <= 1.0
    # monotone in the count: a larger count never gets a smaller feature
    f = np.concatenate([X[:, 0], X[:, 1]])
    cc = np.concatenate([c[i], c[j]])
    o = np.argsort(cc, kind="stable")
    assert (np.diff(f[o]) >= 0).all()
