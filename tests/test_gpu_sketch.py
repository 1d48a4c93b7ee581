"""GPU parity of the per-partition Count-Sketch (Preliminaries; Figure 1)
against the oracle: integer sketches bit-exact (direct exact plans with every
dense tier, on-chip-table plans, UPPER, partition intervals, summary plans
with reserved keys,
streaming calls, reset), real sketches within the fp64 summation bound, the
median estimate over t plans exactly, and the sketch of the full
10,000,000-transaction co-occurrence workload through its Fourier transform
at a few frequencies (a closed form linear in the input)."""
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


def _plan(crp, n_rows, n_cols, P, seeds=(ci.SEED_A, ci.SEED_B), flags=None, **kw):
    f = crp.CRP_PLAN_SKETCH | (crp.CRP_PLAN_DIRECT | crp.CRP_PLAN_DEBUG_CHECKS
                               if flags is None else flags)
    return crp.Plan(n_rows, n_cols, P, seeds[0], seeds[1], flags=f, **kw)


def _random_case(seed, K, n_i, n_j, density, values):
    rng = np.random.default_rng(seed)
    out = []
    for n in (n_i, n_j):
        ptr, idx = [0], []
        for _ in range(K):
            r = rng.random()
            L = 0 if r < 0.1 else (1 if r < 0.2 else (n if r < 0.22 else rng.binomial(n, density)))
            idx.extend(np.sort(rng.choice(n, L, replace=False)).tolist())
            ptr.append(len(idx))
        val = rng.uniform(0.01, 3, len(idx)).astype(np.float32) if values else None
        out.append(O.Compressed(np.array(ptr, np.int64), np.array(idx, np.int32), val, n))
    return out


C1_CONFIGS = [
    dict(P=1), dict(P=64), dict(P=64, groups=8), dict(P=4096),
    dict(P=8192), dict(P=65536, groups=16),          # estimators in HBM (P > 4096)
    dict(P=64, flags=4 | 1 | 2),                     # no warp match
    dict(P=64, hot_items=500), dict(P=256, hot_items=64, warm_items=16),
    dict(P=64, warm_items=100),
    dict(P=64, flags=2), dict(P=8192, groups=4, flags=2),   # on-chip table: added at flush
]


@pytest.mark.parametrize("cfg", C1_CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_c1_sketch_bit_exact(crp, cfg):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.FULL)
    cfg = dict(cfg)
    P = cfg.pop("P")
    plan = _plan(crp, 1000, 1000, P, **cfg)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    want = O.count_sketch(ref, P, ci.SEED_A, ci.SEED_B).astype(np.int64)
    got = plan.sketch()
    assert got.dtype == np.int64 and np.array_equal(got, want)
    # the tables are unchanged by the sketch
    i, j, w, _ = plan.export()
    assert len(i) == len(ref.i) and w.sum() == ref.w.sum()
    plan.close()


def test_c1_upper_sorted_rows_sketch(crp):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc, O.UPPER)
    for flags in (4 | 2, 4 | 16 | 2):   # general enumeration and the i < j enumeration
        plan = _plan(crp, 1000, 1000, 128, flags=flags, mode=crp.CRP_UPPER)
        d = crp.to_device(T)
        plan.accumulate(d, d)
        plan.sync()
        assert np.array_equal(plan.sketch(), O.count_sketch(ref, 128, ci.SEED_A, ci.SEED_B))
        plan.close()


def test_interval_plan_sketches_its_own_partitions(crp):
    # a plan that owns [q, r) enumerates only those terms: its sketch is the
    # oracle's restricted to [q, r), zero elsewhere; the K interval plans of
    # Theorem 1 add up to the whole sketch
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    full = O.count_sketch(O.exact_product(Tc, Tc), 64, ci.SEED_A, ci.SEED_B)
    d = crp.to_device(T)
    total = np.zeros(64, np.int64)
    for q, r in ((0, 16), (16, 40), (40, 64)):
        plan = _plan(crp, 1000, 1000, 64, part_begin=q, part_end=r)
        plan.accumulate(d, d)
        plan.sync()
        got = plan.sketch()
        want = np.zeros(64)
        want[q:r] = full[q:r]
        assert np.array_equal(got, want)
        total += got
        plan.close()
    assert np.array_equal(total, full)


@pytest.mark.parametrize("seed,P,G", [(0, 1, 1), (1, 2, 2), (2, 64, 8), (3, 1024, 32),
                                      (4, 8192, 1), (5, 16, 1)])
def test_random_edge_cases_sketch(crp, seed, P, G):
    A, B = _random_case(seed, 700, 37 + seed * 50, 53 + seed * 30, 0.2, False)
    ref = O.exact_product(A, B, O.FULL)
    plan = _plan(crp, A.n_minor, B.n_minor, P, groups=G, tile_vectors=7)
    plan.accumulate(crp.to_device(A), crp.to_device(B))
    plan.sync()
    assert np.array_equal(plan.sketch(), O.count_sketch(ref, P, ci.SEED_A, ci.SEED_B))
    plan.close()


@pytest.mark.parametrize("seed,P,fl", [(10, 32, None), (11, 8192, None), (12, 64, 2)])
def test_real_sketch_within_summation_bound(crp, seed, P, fl):
    # every term is the exact fp32 product; the fp64 sums differ from the
    # oracle's only in order: |error| <= n eps sum |terms| per estimator
    A, B = _random_case(seed, 600, 80, 90, 0.15, True)
    ref = O.exact_product(A, B, O.FULL)
    plan = _plan(crp, 80, 90, P, value_type=crp.CRP_F32_COMP, flags=fl)
    plan.accumulate(crp.to_device(A), crp.to_device(B))
    plan.sync()
    got = plan.sketch()
    assert got.dtype == np.float64
    want = O.count_sketch(ref, P, ci.SEED_A, ci.SEED_B)
    n = O.total_terms(A, B)
    bound = n * 2.0 ** -52 * np.abs(ref.w).sum()
    np.testing.assert_allclose(got, want, rtol=0, atol=bound)
    plan.close()


def test_signed_values_sketch(crp):
    # Count-Sketch allows signed weights: inputs of both signs, so entries
    # cancel; the bound uses the absolute terms (|a||b| summed per estimator)
    A, B = _random_case(13, 600, 80, 90, 0.15, True)
    rng = np.random.default_rng(99)
    A.val[:] = A.val * np.where(rng.random(len(A.val)) < 0.5, -1, 1).astype(np.float32)
    B.val[:] = B.val * np.where(rng.random(len(B.val)) < 0.5, -1, 1).astype(np.float32)
    ref = O.exact_product(A, B, O.FULL)
    assert (ref.w < 0).any() and (ref.w > 0).any()
    absA = O.Compressed(A.ptr, A.idx, np.abs(A.val), A.n_minor)
    absB = O.Compressed(B.ptr, B.idx, np.abs(B.val), B.n_minor)
    mag = O.exact_product(absA, absB, O.FULL).w.sum()
    for P, fl in ((64, None), (64, 2), (8192, None)):
        plan = _plan(crp, 80, 90, P, value_type=crp.CRP_F32_COMP, flags=fl)
        plan.accumulate(crp.to_device(A), crp.to_device(B))
        plan.sync()
        want = O.count_sketch(ref, P, ci.SEED_A, ci.SEED_B)
        bound = O.total_terms(A, B) * 2.0 ** -52 * mag
        np.testing.assert_allclose(plan.sketch(), want, rtol=0, atol=bound)
        plan.close()


def test_summary_plan_sketch_with_reserved_keys(crp):
    # the summaries drop weight, the sketch does not: in a summary plan with
    # reserved keys (dense block) the sketch is still exact, over two calls
    T = ci.C1.scaled(m=12000).generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc)
    P, ell = 8, 64
    ri, rj, _ = O.topk(ref.i, ref.j, ref.w, 100)
    keys = (ri.astype(np.uint64) << np.uint64(32)) | rj.astype(np.uint64)
    plan = _plan(crp, 1000, 1000, P, flags=0, summary_counters=ell, reserved_counters=128)
    plan.reserve(keys)
    for lo, hi in ((0, 5000), (5000, 12000)):
        part = ci.Sparse(T.ptr[lo:hi + 1] - T.ptr[lo], T.idx[T.ptr[lo]:T.ptr[hi]], None, 1000)
        dd = crp.to_device(part)
        plan.accumulate(dd, dd)
    plan.sync()
    assert np.array_equal(plan.sketch(), O.count_sketch(ref, P, ci.SEED_A, ci.SEED_B))
    plan.close()


def test_streaming_and_reset(crp):
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    want = O.count_sketch(O.exact_product(Tc, Tc), 256, ci.SEED_A, ci.SEED_B)
    plan = _plan(crp, 1000, 1000, 256)
    m = T.n_major // 3
    for lo, hi in ((0, m), (m, T.n_major)):
        part = ci.Sparse(T.ptr[lo:hi + 1] - T.ptr[lo], T.idx[T.ptr[lo]:T.ptr[hi]], None, 1000)
        dd = crp.to_device(part)
        plan.accumulate(dd, dd)
    plan.sync()
    assert np.array_equal(plan.sketch(), want)
    plan.reset()
    assert not plan.sketch().any()
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    assert np.array_equal(plan.sketch(), want)
    plan.close()


@pytest.mark.parametrize("t", [1, 4, 5])
def test_median_estimate_over_instances(crp, t):
    import torch
    T = ci.C1.generate()
    Tc = O.Compressed.of(T)
    ref = O.exact_product(Tc, Tc)
    P = 32
    seeds = [(ci.SEED_A + 2 * r, ci.SEED_B + 2 * r + 1) for r in range(t)]
    d = crp.to_device(T)
    plans = []
    for s in seeds:
        pl = _plan(crp, 1000, 1000, P, seeds=s)
        pl.accumulate(d, d)
        plans.append(pl)
    rng = np.random.default_rng(t)
    top = np.argsort(-ref.w, kind="stable")[:200]
    qi = np.concatenate([ref.i[top], rng.integers(0, 1000, 300)]).astype(np.int32)
    qj = np.concatenate([ref.j[top], rng.integers(0, 1000, 300)]).astype(np.int32)
    got = crp.sketch_estimate(plans, torch.from_numpy(qi).cuda(), torch.from_numpy(qj).cuda())
    ests = [O.sketch_estimate(O.count_sketch(ref, P, *s), qi, qj, P, *s) for s in seeds]
    want = O.sketch_median(ests)
    assert np.array_equal(got.cpu().numpy(), want)
    for pl in plans:
        pl.close()


def test_invalid_uses_are_rejected(crp):
    import torch
    with pytest.raises(crp.CrpError):
        crp.Plan(100, 100, 16, 1, 2, flags=crp.CRP_PLAN_SKETCH | crp.CRP_PLAN_ROUTED)
    plain = crp.Plan(100, 100, 16, 1, 2, flags=crp.CRP_PLAN_DIRECT)
    with pytest.raises(crp.CrpError):
        plain.sketch()
    sk = crp.Plan(100, 100, 16, 1, 2, flags=crp.CRP_PLAN_DIRECT | crp.CRP_PLAN_SKETCH)
    other = crp.Plan(100, 100, 32, 3, 4, flags=crp.CRP_PLAN_DIRECT | crp.CRP_PLAN_SKETCH)
    q = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    bad = torch.tensor([1, 100], dtype=torch.int32, device="cuda")   # 100 >= n_cols
    with pytest.raises(crp.CrpError):
        crp.sketch_estimate([sk, other], q, q)                         # different P
    with pytest.raises(crp.CrpError):
        crp.sketch_estimate([sk, plain], q, q)                         # no sketch
    with pytest.raises(crp.CrpError):
        crp.sketch_estimate([sk], q, bad)
    assert (crp.sketch_estimate([sk], q, q).cpu().numpy() == 0).all()   # nothing accumulated
    for pl in (plain, sk, other):
        pl.close()


def test_full_size_c2_sketch_spectrum(crp):
    # the 10M-transaction workload, direct plan with hot block and warm
    # stripes: the sketch's transform at four frequencies equals the closed
    # form from the inputs (linear in nnz); integer sketch values, so the
    # fp64 transform of either side is accurate to ~1e-9 relative
    T = ci.C2.generate()
    P = 1024
    plan = _plan(crp, T.n_minor, T.n_minor, P, flags=crp.CRP_PLAN_DIRECT, hot_items=2048,
                 warm_items=32, auto_grow=True)
    d = crp.to_device(T)
    plan.accumulate(d, d)
    plan.sync()
    cs = plan.sketch().astype(np.float64)
    L = np.diff(np.asarray(T.ptr)).astype(np.int64)
    assert np.abs(cs).sum() <= float((L * L).sum())
    Tc = O.Compressed.of(T)
    freqs = [0, 1, 37, 511]
    want = O.count_sketch_spectrum(Tc, Tc, P, ci.SEED_A, ci.SEED_B, freqs)
    p = np.arange(P)
    for f, wv in zip(freqs, want):
        got = np.sum(cs * np.exp(2j * np.pi * ((f * p) % P) / P))
        scale = float((L * L).sum())
        assert abs(got - wv) <= 1e-9 * scale, (f, got, wv)
    plan.close()
