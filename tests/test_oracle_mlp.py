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
