"""The tcgen05 heavy-pair predictor against the CPU oracle (same bf16-rounded
operands, fp64 arithmetic), its candidate pairs, its training, and what it
gains in the summary path over the plain summary.

Two kinds of parity, both element by element:

* exact arithmetic: inputs, weights and biases on coarse dyadic grids, so that
  every fp32 sum the kernels form (tensor-core products accumulated in TMEM,
  warp sums, atomics) is exact whatever its order; then every output, every
  gradient element and the loss equal the oracle's fp64 values exactly.
* general random data: an error bound per element from the kernels'
  arithmetic.  Products of bf16 operands are exact in fp32; a sum of n terms
  rounded in fp32 in any order is off by at most 2 n u sum|terms| (u =
  2^-24, a factor 2 allowing truncating adds); a bf16 rounding of a value
  known to within e can go the other way only if the value is within e of a
  rounding midpoint, and then moves it by at most e + one bf16 spacing (one
  possible flip per hidden operand).  These errors are carried forward
  through the network and the backward pass (linear error propagation, in
  fp64 on the host) to a bound for every output and gradient element.  A
  ReLU whose input lies within its error bound of 0 could switch either way;
  such rows are left out of the batch, on both sides.
"""
import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O

pytestmark = pytest.mark.gpu

U = 2.0 ** -24     # fp32 unit roundoff


@pytest.fixture(scope="module")
def crp():
    import torch
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp as c
    torch.cuda.init()
    return c


def _dev(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float32, device="cuda")


# ---------------------------------------------------------------------------
# exact arithmetic
# ---------------------------------------------------------------------------

def _lowest_bit(v):
    """Exponent of the lowest set bit of each nonzero value (fp64)."""
    v = np.abs(np.asarray(v, np.float64)).ravel()
    v = v[v != 0]
    if not len(v):
        return 0
    m, e = np.frexp(v)
    M = np.round(m * 2.0 ** 53).astype(np.int64)
    low = M & -M
    return int((np.log2(low.astype(np.float64)) + e - 53).min())


def _assert_exact_in_f32(terms, axis):
    """Every partial sum of `terms` along `axis`, in any order and grouping,
    is exact in fp32: all terms are multiples of 2^g and the sum of their
    magnitudes is below 2^(24 + g)."""
    g = _lowest_bit(terms)
    S = np.abs(terms).sum(axis=axis)
    assert (S < 2.0 ** (24 + g)).all(), (S.max(), g)


def _exact_case(n, seed):
    """Network and batch on dyadic grids: x, W1 in steps of 1/4 (|x| <= 1,
    |W1| <= 1), b1, b2 in steps of 1/16 (<= 1/2), W2 in steps of 1/8 (<=
    1/4), w3 and b3 in steps of 1/8 (<= 1/2); targets t = y - delta with
    delta in steps of 1/4 (|delta| <= 1), n a power of two."""
    rng = np.random.default_rng(seed)
    d = dict(W1=rng.integers(-4, 5, (64, 2)) / 4, b1=rng.integers(-8, 9, 64) / 16,
             W2=rng.integers(-2, 3, (64, 64)) / 8, b2=rng.integers(-8, 9, 64) / 16,
             w3=rng.integers(-4, 5, 64) / 8, b3=rng.integers(-4, 5, 1) / 8)
    theta = O.mlp_pack(d)
    X = rng.integers(0, 5, (n, 2)) / 4
    y, _ = O.mlp_forward(theta, X)
    t = y - rng.integers(-4, 5, n) / 4
    return theta, X, t


def _check_exact_preconditions(theta, X, t, n_total):
    """The sums of the exact case, checked for exactness in fp32."""
    y, c = O.mlp_forward(theta, X)
    p = c["p"]
    assert np.array_equal(O.bf16_round(p["W1"]), p["W1"])
    assert np.array_equal(O.bf16_round(p["W2"]), p["W2"])
    assert np.array_equal(O.bf16_round(X), X)
    # forward: Z1 (2 products + bias), Z2 (64 products + bias), y (64 fmas + b3)
    _assert_exact_in_f32(np.concatenate([X[:, None, :] * p["W1"][None], np.broadcast_to(
        p["b1"][None, :, None], (len(X), 64, 1))], axis=2), 2)
    assert np.array_equal(O.bf16_round(c["H1b"]), np.maximum(c["Z1"], 0))
    _assert_exact_in_f32(np.concatenate([c["H1b"][:, None, :] * p["W2"][None], np.broadcast_to(
        p["b2"][None, :, None], (len(X), 64, 1))], axis=2), 2)
    H2 = c["H2"]
    _assert_exact_in_f32(np.concatenate([H2 * p["w3"][None], np.full((len(X), 1), p["b3"][0])],
                                        axis=1), 1)
    # backward
    r = y - t
    inv = 1.0 / n_total
    assert np.array_equal(np.float32(t).astype(np.float64), t)
    _assert_exact_in_f32((r * r * inv)[:, None], 0)
    dy = 2 * r * inv
    _assert_exact_in_f32(dy[:, None], 0)
    _assert_exact_in_f32(H2 * dy[:, None], 0)
    dZ2 = np.outer(dy, p["w3"]) * (c["Z2"] > 0)
    assert np.array_equal(O.bf16_round(dZ2), dZ2)
    _assert_exact_in_f32(dZ2, 0)
    _assert_exact_in_f32(dZ2[:, :, None] * c["H1b"][:, None, :], 0)
    _assert_exact_in_f32(dZ2[:, :, None] * p["W2"][None], 1)
    dZ1b = O.bf16_round((dZ2 @ p["W2"]) * (c["Z1"] > 0))
    _assert_exact_in_f32(dZ1b, 0)
    _assert_exact_in_f32(dZ1b[:, :, None] * X[:, None, :], 0)
    return y


@pytest.mark.parametrize("n,seed", [(256, 11), (1024, 12), (128, 13)])
def test_exact_arithmetic_forward_gradient_and_adam(crp, n, seed):
    """Dyadic network and batch: the kernels' outputs, loss and every
    gradient element equal the oracle's exactly.  Two Adam steps match the
    oracle's, run with the kernels' fp32 hyper-parameters, element by
    element: the kernel forms the step with a few fp32 roundings (8 u) from
    bias corrections c = 1 - beta^s that the host rounds to fp32 (an absolute
    error up to 2 u each, relative 2u / c1 and, under the square root,
    u / c2), and rounds the new parameter to fp32 once."""
    import torch
    theta, X, t = _exact_case(n, seed)
    y = _check_exact_preconditions(theta, X, t, n)
    got_y = crp.mlp_forward(_dev(theta), _dev(X)).cpu().numpy().astype(np.float64)
    assert np.array_equal(got_y, y)
    L, g_ref, _ = O.mlp_loss_grad(theta, X, t)
    loss, g = crp.mlp_grad(_dev(theta), _dev(X), _dev(t))
    g = g.cpu().numpy().astype(np.float64)
    assert loss == L
    o = 0
    for name, shape in O.MLP_SIZES:
        k = int(np.prod(shape))
        assert np.array_equal(g[o:o + k], g_ref[o:o + k]), name
        o += k
    assert np.count_nonzero(g_ref) > 1000      # the case exercises most parameters
    # Adam: two steps from zero moments with the exact gradient
    lr = 1e-3
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
    prm, m, v = _dev(theta), torch.zeros(len(theta), device="cuda"), torch.zeros(
        len(theta), device="cuda")
    th, mr, vr = theta.copy(), np.zeros(len(theta)), np.zeros(len(theta))
    for step in (1, 2):
        crp.mlp_adam(prm, m, v, _dev(g_ref), lr, step)
        th_new, mr, vr = O.adam_step(th, mr, vr, g_ref, lr, step, b1=b1, b2=b2)
        got = prm.cpu().numpy().astype(np.float64)
        ulp = np.spacing(np.abs(th_new).astype(np.float32)).astype(np.float64)
        c1, c2 = 1 - b1 ** step, 1 - b2 ** step
        rel = 8 * U + 2 * U / c1 + U / c2
        assert (np.abs(got - th_new) <= ulp + rel * np.abs(th_new - th)).all()
        np.testing.assert_allclose(m.cpu().numpy(), mr, rtol=1e-6, atol=0)
        np.testing.assert_allclose(v.cpu().numpy(), vr, rtol=1e-6, atol=1e-30)
        th = th_new
        g_ref = g_ref * 0.5


# ---------------------------------------------------------------------------
# general random data: element-wise error bounds
# ---------------------------------------------------------------------------

def _bf16_spacing(a):
    """Spacing of bf16 values at |a|: 2^(e-8) for |a| in [2^(e-1), 2^e)."""
    a = np.abs(np.asarray(a, np.float64))
    _, e = np.frexp(a)
    return np.where(a > 0, np.ldexp(1.0, e - 8), 0.0)


def _midpoint_distance(v):
    """Distance of |v| to the nearest bf16 rounding boundary (0 at 0)."""
    a = np.abs(np.asarray(v, np.float64))
    _, e = np.frexp(a)
    sp = np.ldexp(1.0, e - 8)
    base = np.ldexp(1.0, e - 1)                 # first bf16 value of the binade
    d_in = np.abs(np.mod((a - base) / sp, 1.0) - 0.5) * sp
    d_below = a - base + sp / 4                 # midpoint under the binade start
    return np.where(a > 0, np.minimum(d_in, d_below), 0.0)


def _rounding_deviation(v, e):
    """Largest |bf16(v') - bf16(v)| over |v' - v| <= e: 0 unless v is within
    e of a rounding midpoint, else e plus one spacing."""
    flip = _midpoint_distance(v) <= e
    return np.where(flip, e + _bf16_spacing(np.abs(v) + e), 0.0)


def _error_model(theta, X, t, n_total):
    """Oracle values and, per row and element, bounds on how far the
    kernels' fp32 values can be from them.  Returns (rows whose ReLU
    decisions are uncertain, dict of oracle values and bounds)."""
    y, c = O.mlp_forward(theta, X)
    p = c["p"]
    Xb, W1b, Z1, H1b, W2b, Z2, H2 = (c[k] for k in ("Xb", "W1b", "Z1", "H1b", "W2b", "Z2", "H2"))
    aW1, aW2, aw3 = np.abs(W1b), np.abs(W2b), np.abs(p["w3"])
    # forward: Z1 = x W1^T + b1 (2 products, the bias), Z2 = H1 W2^T + b2 (64
    # products, the bias), y = b3 + sum H2 w3 (64 fmas)
    eZ1 = 2 * U * 4 * (np.abs(Xb) @ aW1.T + np.abs(p["b1"]))
    amb = (np.abs(Z1) <= eZ1).any(axis=1)
    mask1 = Z1 > 0
    dH1b = _rounding_deviation(np.maximum(Z1, 0.0), eZ1) * mask1
    eZ2 = 2 * U * 66 * (np.abs(H1b) @ aW2.T + np.abs(p["b2"])) + dH1b @ aW2.T
    amb |= (np.abs(Z2) <= eZ2).any(axis=1)
    mask2 = Z2 > 0
    eH2 = eZ2 * mask2
    ey = eH2 @ aw3 + 2 * U * 66 * (abs(p["b3"][0]) + H2 @ aw3)
    # backward: r = y - t, dy = 2 r / n_total, dZ2 = dy w3 (masked, to bf16),
    # dH1 = dZ2 W2 (64 products), dZ1 = dH1 (masked, to bf16)
    inv = 1.0 / n_total
    r = y - t
    er = ey + U * np.abs(r)
    dy = 2 * r * inv
    edy = 2 * inv * er + U * np.abs(dy)
    dZ2 = np.outer(dy, p["w3"]) * mask2
    edZ2 = (np.outer(edy, aw3) + U * np.abs(dZ2)) * mask2
    dZ2b = O.bf16_round(dZ2)
    ddZ2b = _rounding_deviation(dZ2, edZ2) * mask2
    dZ1 = (dZ2b @ W2b) * mask1
    edH1 = (2 * U * 66 * (np.abs(dZ2b) @ aW2) + ddZ2b @ aW2) * mask1
    dZ1b = O.bf16_round(dZ1)
    ddZ1b = _rounding_deviation(dZ1, edH1) * mask1
    return amb, dict(y=y, ey=ey, r=r, er=er, dy=dy, edy=edy, H2=H2, eH2=eH2, Xb=Xb, H1b=H1b,
                     dH1b=dH1b, dZ2b=dZ2b, ddZ2b=ddZ2b, dZ1b=dZ1b, ddZ1b=ddZ1b, inv=inv)


def _gradient_bounds(m):
    """Bound per parameter (layout of the oracle's gradient) and for the loss,
    from the row bounds of _error_model: each gradient element is a sum over
    rows of products whose factors are known to within their bounds, summed
    in fp32 in some order."""
    n = len(m["y"])
    acc = 2 * U * (n + 64)
    aX, aH1, adZ2, adZ1 = np.abs(m["Xb"]), np.abs(m["H1b"]), np.abs(m["dZ2b"]), np.abs(m["dZ1b"])
    ady = np.abs(m["dy"])
    bW1 = m["ddZ1b"].T @ aX + acc * (adZ1.T @ aX)
    bb1 = m["ddZ1b"].sum(0) + acc * adZ1.sum(0)
    bW2 = (m["ddZ2b"].T @ aH1 + adZ2.T @ m["dH1b"] + m["ddZ2b"].T @ m["dH1b"]
           + acc * (adZ2.T @ aH1))
    bb2 = m["ddZ2b"].sum(0) + acc * adZ2.sum(0)
    bw3 = m["eH2"].T @ ady + m["H2"].T @ m["edy"] + m["eH2"].T @ m["edy"] + acc * (m["H2"].T @ ady)
    bb3 = np.array([m["edy"].sum() + acc * ady.sum()])
    bL = ((2 * np.abs(m["r"]) * m["er"] + m["er"] ** 2) * m["inv"]).sum() + acc * (
        m["r"] ** 2 * m["inv"]).sum()
    return O.mlp_pack(dict(W1=bW1, b1=bb1, W2=bW2, b2=bb2, w3=bw3, b3=bb3)), bL


@pytest.mark.parametrize("n,seed", [(1000, 0), (128, 1), (1, 2), (4099, 3)])
def test_forward_matches_oracle_elementwise(crp, n, seed):
    rng = np.random.default_rng(seed)
    theta = O.mlp_init(seed)
    X = rng.uniform(0, 1, (n, 2)).astype(np.float32).astype(np.float64)
    amb, m = _error_model(theta, X, np.zeros(n), n)
    assert amb.sum() <= max(1, n // 100), amb.sum()
    keep = ~amb
    got = crp.mlp_forward(_dev(theta), _dev(X[keep])).cpu().numpy().astype(np.float64)
    err = np.abs(got - m["y"][keep])
    assert (err <= m["ey"][keep]).all(), (err - m["ey"][keep]).max()
    # the bounds are tight enough to mean something: the median bound is under
    # 1e-3 of the output (worst-case summation bounds of 64-term sums)
    assert np.median(m["ey"][keep] / np.maximum(np.abs(m["y"][keep]), 1e-3)) < 1e-3


@pytest.mark.parametrize("n,seed", [(1000, 4), (300, 5), (4096, 6)])
def test_gradient_matches_oracle_elementwise(crp, n, seed):
    rng = np.random.default_rng(seed)
    theta = O.mlp_init(seed)
    X = rng.uniform(0, 1, (n, 2)).astype(np.float32).astype(np.float64)
    t = rng.uniform(0, 2, n).astype(np.float32).astype(np.float64)
    amb, _ = _error_model(theta, X, t, n)
    assert amb.sum() <= max(1, n // 100), amb.sum()
    keep = ~amb
    Xk, tk = X[keep], t[keep]
    L, g_ref, _ = O.mlp_loss_grad(theta, Xk, tk, n_total=n)
    _, m = _error_model(theta, Xk, tk, n)
    bound, bL = _gradient_bounds(m)
    loss, g = crp.mlp_grad(_dev(theta), _dev(Xk), _dev(tk), n_total=n)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - L) <= bL + U * abs(L)
    o = 0
    for name, shape in O.MLP_SIZES:
        k = int(np.prod(shape))
        d = np.abs(g[o:o + k] - g_ref[o:o + k])
        b = bound[o:o + k] + U * np.abs(g_ref[o:o + k])     # the final fp32 value
        assert (d <= b).all(), (name, int(np.argmax(d - b)), (d - b).max())
        o += k
    # not vacuous: over the whole gradient the bounds are a small fraction of it
    assert bound.sum() < 0.01 * np.abs(g_ref).sum(), bound.sum() / np.abs(g_ref).sum()


@pytest.mark.parametrize("R", [64, 257])
def test_candidate_pairs_match_oracle(crp, R):
    """crp_candidate_pairs against the oracle: the prefix item counts, the R
    items of largest count (items above the R-th count must all be there; of
    the items tied at it, any), every pair i < j of them once, and the
    features log(1 + c) / log(1 + max c) element by element (fp32 logf within
    a few ulps: relative 1e-6; log(1) = 0 exactly)."""
    T = _stream(3030, 40_000, 5_000)
    pre = _prefix(T, 0.05)
    Pc = O.Compressed.of(pre)
    c = O.prefix_item_counts(Pc)
    i, j, x = crp.candidate_pairs(crp.to_device(pre), T.n_minor, R)
    i = i.cpu().numpy().astype(np.int64)
    j = j.cpu().numpy().astype(np.int64)
    x = x.cpu().numpy().astype(np.float64)
    assert len(i) == R * (R - 1) // 2
    assert (i < j).all()
    keys = i * T.n_minor + j
    assert len(np.unique(keys)) == len(keys)
    items = np.unique(np.concatenate([i, j]))
    assert len(items) == R
    thr = np.sort(c)[::-1][R - 1]                 # the R-th largest count
    assert set(np.flatnonzero(c > thr).tolist()) <= set(items.tolist())
    assert (c[items] >= thr).all()
    a, b = np.triu_indices(R, k=1)
    want_keys = np.sort(items[a] * T.n_minor + items[b])
    assert np.array_equal(np.sort(keys), want_keys)
    # the oracle's own candidates agree wherever the choice is unique
    oi, oj, oX, _ = O.candidate_pairs(Pc, R)
    top = set(np.flatnonzero(c > thr).tolist())
    sel = np.array([u in top and v in top for u, v in zip(oi.tolist(), oj.tolist())])
    o_keys = oi[sel] * T.n_minor + oj[sel]
    pos = np.searchsorted(np.sort(keys), o_keys)
    assert np.array_equal(np.sort(keys)[pos], o_keys)
    want = O.marginal_features(c[i], c[j], np.log1p(c.max()))
    np.testing.assert_allclose(x, want, rtol=1e-6, atol=0)

def test_training_reduces_loss(crp):
    rng = np.random.default_rng(9)
    X = rng.uniform(0, 1, (4096, 2))
    t = np.sin(3 * X[:, 0]) + X[:, 1] ** 2          # a smooth target
    theta = _dev(O.mlp_init(9))
    tr = crp.MLPTrainer(theta, lr=1e-2)
    dX, dt = _dev(X), _dev(t)
    first = tr.step(dX, dt)
    for _ in range(300):
        last = tr.step(dX, dt)
    assert last < 0.1 * first, (first, last)


def _stream(seed, m, n):
    # the heavy-entry recipe (Poisson(15) lengths, Zipf(1.2) items), scaled
    return ci.transactions(seed, m, n, 15.0, 0, -1, 1.2)


def _prefix(T, frac=0.01):
    m = max(1, int(T.n_major * frac))
    return ci.Sparse(T.ptr[:m + 1], T.idx[:T.ptr[m]], None, T.n_minor)


def _train_predictor(crp, R):
    """Labels: exact pair counts (oracle) of a training stream; features:
    prefix marginals of the candidate pairs (the library's own candidates)."""
    T = _stream(2024, 60_000, 20_000)
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.UPPER)
    cnt = dict(zip((ref.i * T.n_minor + ref.j).tolist(), ref.w.tolist()))
    i, j, x = crp.candidate_pairs(crp.to_device(_prefix(T)), T.n_minor, R)
    keys = (i.cpu().numpy().astype(np.int64) * T.n_minor + j.cpu().numpy())
    y = np.log1p(np.array([cnt.get(int(k), 0.0) for k in keys]))
    scale = y.max()
    theta = _dev(O.mlp_init(7))
    tr = crp.MLPTrainer(theta, lr=3e-3)
    ty = _dev(y / scale)
    losses = [tr.step(x, ty) for _ in range(400)]
    assert losses[-1] < 0.5 * losses[0]
    return theta


@pytest.fixture(scope="module")
def trained(crp):
    return _train_predictor(crp, 256)


@pytest.mark.parametrize("ell,k", [(64, 100), (256, 1000), (1024, 1000)])
def test_predictor_gain_over_plain_summary(crp, trained, ell, k):
    """Summary-mode top-k weight error (vs the exact oracle) with the network
    reserving 2048 exact counters, against the plain summary and against
    reserving by the product of marginals.  Regimes: lossy (ell = 64, k = 100;
    ell = 256, k = 1000) and ample counters (ell = 1024)."""
    R, n_res, P = 256, 2048, 16
    T = _stream(77, 60_000, 20_000)
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.UPPER)
    true = dict(zip((ref.i * T.n_minor + ref.j).tolist(), ref.w.tolist()))
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k, upper_only=True)
    d = crp.to_device(T)
    pre = crp.to_device(_prefix(T))

    def run(params, reserve):
        plan = crp.Plan(T.n_minor, T.n_minor, P, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER,
                        summary_counters=ell, reserved_counters=n_res if reserve else 0)
        if reserve:
            crp.predict_reserve(plan, pre, T.n_minor, params, R, n_res)
        plan.accumulate(d, d)
        plan.sync()
        ti, tj, tw, _ = plan.topk(k, upper=True)
        plan.close()
        got = sum(true.get(int(a) * T.n_minor + int(b), 0.0) for a, b in zip(ti, tj))
        return 1.0 - got / rw.sum()

    err_plain = run(None, False)
    err_mlp = run(trained, True)
    err_heur = run(None, True)
    print(f"ell={ell} top-{k} weight error: plain {err_plain:.4f}, predictor {err_mlp:.4f}, "
          f"product-of-marginals {err_heur:.4f}")
    assert err_mlp <= err_plain + 1e-9
