"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
reference outputs, exhaustive enumeration, dense matrix products (numpy),
closed forms and the Space-Saving guarantees (Preliminaries).
"""
import itertools
import os

import numpy as np
import pytest

import crp_inputs as ci
from oracle import crp_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sparse(rng, K, n, density, values=True, forced=()):
    """Random compressed matrix with K vectors over [n]; ``forced`` lists
    (k, length) overrides, used for empty, singleton and dense vectors."""
    ptr = [0]
    idx = []
    lens = {k: L for k, L in forced}
    for k in range(K):
        L = lens.get(k, rng.binomial(n, density))
        sel = np.sort(rng.choice(n, size=L, replace=False))
        idx.extend(sel.tolist())
        ptr.append(len(idx))
    val = rng.uniform(0.1, 2.0, size=len(idx)).astype(np.float32) if values else None
    return O.Compressed(np.array(ptr, np.int64), np.array(idx, np.int32), val, n)


# ---------------------------------------------------------------------------
# Hash family
# ---------------------------------------------------------------------------

def test_splitmix64_reference_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    assert O.splitmix64(0, 3) == want


@pytest.mark.parametrize("lbits", [1, 2, 3, 5])
def test_multiply_add_shift_is_pairwise_independent_exhaustively(lbits):
    # Dietzfelbinger's multiply-add-shift: 4-bit keys, 8-bit words (8 >= 4 +
    # l - 1); over all (a, b) every pair of outputs for two distinct keys is
    # equally likely -- the pairwise independence Lemma 1 asks for.
    w, kb = 8, 4
    a, b = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    a = a.ravel()
    b = b.ravel()

    def h(x):
        return (((a * x) + b) & 255) >> (w - lbits)

    for x, y in itertools.combinations(range(1 << kb), 2):
        joint = h(x) * (1 << lbits) + h(y)
        counts = np.bincount(joint, minlength=1 << (2 * lbits))
        assert (counts == 65536 >> (2 * lbits)).all(), (x, y)
        # the scalar oracle hash is the same map at this width
    for x in range(16):
        for aa, bb in [(3, 7), (255, 0), (128, 129)]:
            want = (((aa * x) + bb) & 255) >> (w - lbits)
            assert O.mas_hash_scalar(x, aa, bb, lbits, word_bits=8) == want


def test_side_hash_64bit_matches_scalar_definition():
    rng = np.random.default_rng(5)
    xs = rng.integers(0, 2**31, size=200)
    for seed in (1, ci.SEED_A, ci.SEED_B):
        a, b = O.hash_params(seed)
        for lg in (0, 1, 6, 13, 16):
            got = O.side_hash(xs, seed, lg)
            want = [O.mas_hash_scalar(int(x), a, b, lg) for x in xs]
            assert got.tolist() == want


def test_partition_hash_range_and_P1():
    rng = np.random.default_rng(1)
    i = rng.integers(0, 10**6, 5000)
    j = rng.integers(0, 10**6, 5000)
    assert (O.partition_of(i, j, 1, 1, 2) == 0).all()
    for P in (2, 64, 8192):
        p = O.partition_of(i, j, P, ci.SEED_A, ci.SEED_B)
        assert p.min() >= 0 and p.max() < P
    with pytest.raises(ValueError):
        O.partition_of(i, j, 48, 1, 2)


def test_partition_hash_is_close_to_uniform_on_entries():
    # h(i,j) = h_a(i) + h_b(j) mod P is pairwise independent (Lemma 1 proof),
    # so over a grid of distinct entries each bucket gets ~1/P of them.
    ii, jj = np.meshgrid(np.arange(300), np.arange(300), indexing="ij")
    P = 16
    p = O.partition_of(ii.ravel(), jj.ravel(), P, ci.SEED_A, ci.SEED_B)
    c = np.bincount(p, minlength=P)
    exp = ii.size / P
    chi2 = ((c - exp) ** 2 / exp).sum()
    assert chi2 < 60  # 15 d.o.f.; p ~ 1e-6 threshold


GAMMA = 0x9E3779B97F4A7C15


def test_partition_hash_worked_values():
    # hand-worked from the published SplitMix64 outputs (golden fixture)
    rows = [l.strip().split("|") for l in open(os.path.join(GOLD, "partition_hash_worked.txt"))
            if l.strip() and not l.startswith("#")]
    n = 0
    for r in rows:
        if r[0] == "S":
            P, x, ha, hb = map(int, r[1:])
            lg = P.bit_length() - 1
            assert int(O.side_hash(np.array([x]), 0, lg)[0]) == ha
            assert int(O.side_hash(np.array([x]), GAMMA, lg)[0]) == hb
        else:
            P, i, j, h = map(int, r[1:])
            assert int(O.partition_of(np.array([i]), np.array([j]), P, 0, GAMMA)[0]) == h
        n += 1
    assert n == 23


@pytest.mark.parametrize("P", [2, 8, 64, 4096])
@pytest.mark.parametrize("seeds", [(ci.SEED_A, ci.SEED_B), (1, 2), (0, GAMMA)])
def test_partition_hash_is_additive_mod_P(P, seeds):
    # Lemma 1's cyclic windows rest on h(i,j) = h_a(i) + h_b(j) mod P: for two
    # rows i1, i2 the difference h(i1, j) - h(i2, j) mod P is the same for every
    # column j and equals h_a(i1) - h_a(i2); likewise for two columns.  XOR,
    # subtraction or a swapped side would break one of the two identities.
    sa, sb = seeds
    lg = P.bit_length() - 1
    rng = np.random.default_rng(P)
    i = rng.integers(0, 2**31, 40)
    j = rng.integers(0, 2**31, 250)
    H = O.partition_of(i[:, None], j[None, :], P, sa, sb)
    ha = np.array([O.mas_hash_scalar(int(x), *O.hash_params(sa), lg) for x in i])
    hb = np.array([O.mas_hash_scalar(int(x), *O.hash_params(sb), lg) for x in j])
    rows = (H - H[:1, :]) % P
    assert (rows == ((ha - ha[0]) % P)[:, None]).all()
    cols = (H - H[:, :1]) % P
    assert (cols == ((hb - hb[0]) % P)[None, :]).all()
    # every pair against the scalar definition
    for x in range(0, len(i), 7):
        for y in range(0, len(j), 11):
            assert H[x, y] == (int(ha[x]) + int(hb[y])) % P


# ---------------------------------------------------------------------------
# Exact product: dense brute force and closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_exact_product_equals_dense_matmul(seed):
    rng = np.random.default_rng(seed)
    n_i, n_j, K = int(rng.integers(1, 64)), int(rng.integers(1, 64)), int(rng.integers(1, 200))
    forced = [(0, 0), (1 % K, 1), (2 % K, n_i)]
    A = _rand_sparse(rng, K, n_i, 0.1, True, forced)
    forced_b = [(0, n_j), (1 % K, 0), (3 % K, 1)]
    B = _rand_sparse(rng, K, n_j, 0.1, True, forced_b)
    want = O.dense(A).T @ O.dense(B)
    got = O.exact_product(A, B, O.FULL, chunk_terms=97)
    D = np.zeros((n_i, n_j))
    D[got.i, got.j] = got.w
    np.testing.assert_allclose(D, want, rtol=1e-12, atol=0)
    nz = want != 0
    assert nz.sum() == len(got.i)
    assert got.terms == O.total_terms(A, B)


@pytest.mark.parametrize("seed", range(3))
def test_exact_product_equals_loop_definition(seed):
    rng = np.random.default_rng(100 + seed)
    A = _rand_sparse(rng, 40, 20, 0.3, True, [(0, 0), (1, 20)])
    B = _rand_sparse(rng, 40, 25, 0.3, True, [(2, 0), (3, 1)])
    for mode in (O.FULL, O.UPPER):
        loop = O.exact_product_loop(A, B, mode)
        vec = O.exact_product(A, B, mode).as_dict()
        assert loop.keys() == vec.keys()
        for k in loop:
            assert abs(loop[k] - vec[k]) <= 1e-12 * abs(loop[k])


def _tx(seed, m, n, lam, lmin, lmax, s):
    T = ci.transactions(seed, m, n, lam, lmin, lmax, s)
    return O.Compressed.of(T)


def test_cooccurrence_closed_forms():
    T = _tx(7, 3000, 200, 8.0, 0, 30, 1.1)
    # duplicate transactions, as real streams have
    T = O.Compressed(np.concatenate([T.ptr, T.ptr[-1] + T.ptr[1:11] - T.ptr[0]]),
                     np.concatenate([T.idx, T.idx[: T.ptr[10]]]), None, T.n_minor)
    L = np.diff(T.ptr)
    full = O.exact_product(T, T, O.FULL)
    # total weight = sum_k |a_k||b_k| = sum L^2 (FULL); L(L-1)/2 above the diagonal
    assert full.w.sum() == (L * L).sum() == full.terms
    upper = O.exact_product(T, T, O.UPPER)
    assert upper.w.sum() == (L * (L - 1) // 2).sum() == upper.terms
    # the diagonal holds the support of each item
    d = full.i == full.j
    support = np.bincount(T.idx, minlength=T.n_minor)
    assert (full.w[d] == support[full.i[d]]).all()
    assert d.sum() == (support > 0).sum()
    # symmetry of T^T T
    fd = full.as_dict()
    for (a, b), w in fd.items():
        assert fd[(b, a)] == w
    # upper = the i<j half of full
    ud = upper.as_dict()
    assert ud == {k: v for k, v in fd.items() if k[0] < k[1]}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_entries_are_bounded_by_row_and_column_degrees(seed):
    # for {0,1} inputs C(i,j) = #{k : i in a_k and j in b_k} <= min(deg_A(i),
    # deg_B(j)), with equality when one item always occurs with the other: the
    # bound the top-k uses to answer from the pairs of frequent items
    rng = np.random.default_rng(seed)
    A = _rand_sparse(rng, 300, 40, 0.15, values=False)
    B = _rand_sparse(rng, 300, 50, 0.15, values=False)
    prod = O.exact_product(A, B, O.FULL)
    deg_a = np.bincount(A.idx, minlength=A.n_minor)
    deg_b = np.bincount(B.idx, minlength=B.n_minor)
    assert (prod.w <= np.minimum(deg_a[prod.i], deg_b[prod.j])).all()
    # tight case: every vector of B holds item 0, so C(i, 0) = deg_A(i)
    rows = [np.union1d([0], B.idx[B.ptr[k]:B.ptr[k + 1]]) for k in range(B.n_major)]
    B0 = O.Compressed(np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64),
                      np.concatenate(rows).astype(np.int32), None, B.n_minor)
    p0 = O.exact_product(A, B0, O.FULL)
    col0 = p0.j == 0
    assert np.array_equal(p0.w[col0], deg_a[p0.i[col0]].astype(float))


def test_entry_definition_matches_product():
    T = _tx(9, 2000, 150, 6.0, 1, 20, 1.0)
    full = O.exact_product(T, T, O.FULL)
    cols = O.Compressed.of(ci.transpose(ci.Sparse(T.ptr, T.idx, None, T.n_minor)))
    rng = np.random.default_rng(0)
    for q in rng.integers(0, len(full.i), 50):
        assert O.entry(cols, cols, int(full.i[q]), int(full.j[q])) == full.w[q]


# ---------------------------------------------------------------------------
# Consistent partitioning and Lemma 1
# ---------------------------------------------------------------------------

def test_interval_terms_cover_outer_product_disjointly():
    rng = np.random.default_rng(3)
    P = 16
    for trial in range(5):
        a = np.sort(rng.choice(100, 12, replace=False))
        b = np.sort(rng.choice(100, 9, replace=False))
        va = rng.uniform(1, 2, len(a))
        vb = rng.uniform(1, 2, len(b))
        cuts = sorted(set([0, P] + rng.integers(1, P, 3).tolist()))
        got = []
        for q, r in zip(cuts[:-1], cuts[1:]):
            part = O.interval_terms(a, va, b, vb, q, r, P, ci.SEED_A, ci.SEED_B)
            for (i, j, w) in part:
                h = int(O.partition_of(np.array([i]), np.array([j]), P, ci.SEED_A,
                                       ci.SEED_B)[0])
                assert q <= h < r
            got.extend(part)
        assert len(got) == len(a) * len(b)
        assert sorted((i, j) for i, j, _ in got) == sorted(
            (int(x), int(y)) for x in a for y in b)


def test_split_by_partition_is_a_partition():
    T = _tx(11, 1000, 120, 6.0, 1, 20, 1.0)
    full = O.exact_product(T, T, O.FULL)
    parts = O.split_by_partition(full, 8, ci.SEED_A, ci.SEED_B)
    assert sum(len(p.i) for p in parts) == len(full.i)
    keys = np.concatenate([p.keys() for p in parts])
    assert len(np.unique(keys)) == len(keys)
    for q, p in enumerate(parts):
        assert (O.partition_of(p.i, p.j, 8, ci.SEED_A, ci.SEED_B) == q).all()
    terms = O.partition_term_counts(T, T, 8, ci.SEED_A, ci.SEED_B)
    assert [int(p.w.sum()) for p in parts] == terms.tolist()


def test_load_balance_theorem1():
    # Theorem 1: the number of entries of one outer product landing in a
    # processor's interval has variance <= its mean W = |a||b|/K.
    rng = np.random.default_rng(4)
    K = 8
    P = 64
    a = np.sort(rng.choice(10**6, 120, replace=False))
    b = np.sort(rng.choice(10**6, 150, replace=False))
    counts = []
    for s in range(300):
        sa, sb = O.splitmix64(s, 2)
        p = O.partition_of(np.repeat(a, len(b)), np.tile(b, len(a)), P, sa, sb)
        counts.append(np.bincount(p * K // P, minlength=K))
    counts = np.array(counts, dtype=float)
    W = len(a) * len(b) / K
    assert abs(counts.mean() - W) < 1e-9
    assert counts.var(axis=0).max() <= 1.25 * W


# ---------------------------------------------------------------------------
# Space-Saving
# ---------------------------------------------------------------------------

def _golden_ss():
    rows = []
    for line in open(os.path.join(GOLD, "space_saving_worked.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, ell, stream, final = line.strip().split("|")
        st = [(int(k), int(w)) for k, w in (x.split(":") for x in stream.split(","))]
        fin = {int(k): (int(c), int(o)) for k, c, o in (x.split(":") for x in final.split(","))}
        rows.append((int(ell), st, fin))
    return rows


def test_space_saving_worked_examples():
    for ell, stream, final in _golden_ss():
        assert O.space_saving(stream, ell) == final


@pytest.mark.parametrize("ell", [1, 4, 16, 64])
def test_space_saving_guarantees(ell):
    rng = np.random.default_rng(ell)
    keys = (rng.zipf(1.3, 4000) % 300).tolist()
    ws = rng.integers(1, 4, len(keys)).tolist()
    stream = list(zip(keys, ws))
    true: dict = {}
    for k, w in stream:
        true[k] = true.get(k, 0) + w
    W = sum(ws)
    s = O.space_saving(stream, ell)
    assert len(s) == min(ell, len(true))
    mn = min(c for c, _ in s.values())
    for k, (c, o) in s.items():
        assert c - o <= true[k] <= c
        assert o <= W / ell
    for k, t in true.items():
        if t > W / ell:
            assert k in s
        if k not in s:
            assert t <= mn
    assert sum(c for c, _ in s.values()) == W  # the summary is full


def test_space_saving_exact_when_counters_suffice():
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 50, 3000).tolist()
    stream = [(k, 1) for k in keys]
    s = O.space_saving(stream, 50)
    assert {k: c for k, (c, o) in s.items()} == {k: keys.count(k) for k in set(keys)}
    assert all(o == 0 for _, o in s.values())


# ---------------------------------------------------------------------------
# Top-k
# ---------------------------------------------------------------------------

def test_topk_order_and_ties():
    i = np.array([5, 1, 1, 2, 0, 3])
    j = np.array([0, 2, 1, 9, 4, 3])
    w = np.array([7., 7., 7., 9., 1., 7.])
    ti, tj, tw = O.topk(i, j, w, 4)
    assert list(zip(ti, tj, tw)) == [(2, 9, 9.), (1, 1, 7.), (1, 2, 7.), (3, 3, 7.)]
    ti, tj, tw = O.topk(i, j, w, 10, upper_only=True)
    assert list(zip(ti, tj)) == [(2, 9), (1, 2), (0, 4)]


@pytest.mark.parametrize("k,n_hot", [(10, 16), (100, 64), (1000, 8), (1000, 4096)])
def test_certified_topk_pairs_equals_brute_force(k, n_hot):
    # against the whole exact product (UPPER) and its top k; n_hot = 8 cannot
    # certify 1000 pairs, so the hot set grows until it does
    T = O.Compressed.of(ci.C1.scaled(m=6000).generate())
    ref = O.exact_product(T, T, O.UPPER)
    ri, rj, rw = O.topk(ref.i, ref.j, ref.w, k)
    gi, gj, gw, cert = O.certified_topk_pairs(T, k, n_hot, chunk=1000)
    assert gi.tolist() == ri.tolist() and gj.tolist() == rj.tolist() and gw.tolist() == rw.tolist()
    assert cert["kth"] > cert["bound"] or cert["n_hot"] >= T.n_minor
    assert cert["n_hot"] >= min(n_hot, T.n_minor)


@pytest.mark.parametrize("P,values", [(64, False), (8, True), (1, False), (1024, False)])
def test_partition_entries_equal_the_split_product(P, values):
    # every partition's entries, found by the side-hash join, against the
    # whole product split by partition (and, with values, the fp64 sums)
    if values:
        rng = np.random.default_rng(3)
        A = _rand_sparse(rng, 300, 40, 0.2, True, [(0, 0), (1, 40)])
        B = _rand_sparse(rng, 300, 50, 0.2, True, [(0, 50), (2, 0)])
    else:
        A = B = O.Compressed.of(ci.C1.scaled(m=3000).generate())
    parts = O.split_by_partition(O.exact_product(A, B, O.FULL), P, ci.SEED_A, ci.SEED_B)
    for p in sorted(set([0, P - 1, P // 3, P // 2])):
        got = O.partition_entries(A, B, P, p, ci.SEED_A, ci.SEED_B, chunk=777)
        want = parts[p]
        assert got.i.tolist() == want.i.tolist() and got.j.tolist() == want.j.tolist()
        np.testing.assert_allclose(got.w, want.w, rtol=1e-12, atol=0)
