"""CPU oracle for the column-row partitioned sparse product (CRoP).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It is a
plain, slow, single-threaded restatement of what the product computes, written
from the paper (Campagna, Kutzkov, Pagh, "On Parallelizing Matrix
Multiplication by the Column-Row Method"), and it shares no code with the CUDA
path: the hash, the enumeration, the accumulation and the summaries are all
written out again here.  Floating point is fp64.

Sections of the paper each function follows:

* Preliminaries, Notation: ``C = A B = sum_k a_k b_k``; the weight of entry
  (i, j) is ``sum_k a_k(i) b_k(j)``; ``[n] = {0..n-1}``
  -> :func:`outer_product_terms`, :func:`exact_product_loop`,
  :func:`exact_product`, :func:`entry`.
* Section 4, Lemma 1 (proof): ``h(i,j) = (h_a(i) + h_b(j)) mod P`` with
  pairwise independent ``h_a, h_b``; the set ``E_L^{ab}`` of entries of the
  outer product ``ab`` hashing into an interval ``L = [q, r)``
  -> :func:`hash_params`, :func:`side_hash`, :func:`partition_of`,
  :func:`interval_terms` (tests every pair; it does not use the two-pointer
  scan, so that scan is checked against the definition),
  :func:`partition_entries` (one partition's entries of a large product).
* Preliminaries, Space-Saving, with weighted positive updates
  -> :func:`space_saving`; one summary per bucket (Figure 1, Section 6's
  many-bucket regime) -> :func:`partition_streams`, :func:`bucket_summaries`.
* Preliminaries, Count-Sketch, and Figure 1 (``CS[h(e)] += e s(e)``); the
  median of t instances
  -> :func:`side_sign`, :func:`sign_of`, :func:`count_sketch_terms`,
  :func:`count_sketch`, :func:`count_sketch_spectrum`, :func:`sketch_estimate`,
  :func:`sketch_median`.
* Section 6 (case study): support of a pair = number of transactions holding
  it, i.e. the entries above the diagonal of ``T^T T``; heaviest entries
  -> :func:`topk`; the heaviest pairs of a large ``T^T T`` from the exact
  counts of the pairs of frequent items and the support bound
  -> :func:`certified_topk_pairs`.
* Not in the paper: the heavy-pair predictor (a 2 -> 64 -> 64 -> 1 network
  on the marginal counts of a prefix) -> :func:`mlp_forward`,
  :func:`mlp_loss_grad`, :func:`adam_step`, :func:`prefix_item_counts`,
  :func:`top_items`, :func:`candidate_pairs`, :func:`marginal_features`.

Readings where the paper is silent:

* Hash family: the paper requires pairwise independence only.  ``(a, b)`` are
  the first two SplitMix64 outputs (Steele, Lea, Flood 2014) from the seed, and
  ``h(x) = ((a x + b) mod 2^64) >> (64 - log2 P)`` (Dietzfelbinger's
  multiply-add-shift); ``P`` is a power of two; ``P = 1`` maps everything to 0.
* Space-Saving ties: the slot evicted is the one of minimum count, ties broken
  by the smallest key (i, j); a weighted insert of weight w into a full summary
  takes ``(key, min + w, min)``.
* Top-k order: weight descending, then i ascending, then j ascending.
* Sign hash of an entry: ``s(i, j) = s_a(i) s_b(j)`` with ``s_x(v) = +1`` or
  ``-1`` from the top bit of a multiply-add hash whose ``(c, d)`` are the third
  and fourth SplitMix64 outputs of the side's seed (pairwise independent over
  pairs when the side hashes are); one estimator per partition.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
FULL = 0   # every entry (i, j)
UPPER = 1  # only entries above the diagonal, i < j (pair mining, Section 6)


# ---------------------------------------------------------------------------
# Hashing (Lemma 1 proof; Preliminaries: k-wise independence)
# ---------------------------------------------------------------------------

def splitmix64(seed: int, count: int) -> list[int]:
    """The first ``count`` outputs of SplitMix64 started from state ``seed``
    (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
    OOPSLA 2014): the state advances by the golden-gamma constant and each
    output is the state passed through the variant-13 mixer."""
    out = []
    x = seed & MASK64
    for _ in range(count):
        x = (x + 0x9E3779B97F4A7C15) & MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        out.append(z ^ (z >> 31))
    return out


def hash_params(seed: int) -> tuple[int, int]:
    """Multiplier and addend of one side hash, drawn from ``seed``."""
    a, b = splitmix64(seed, 2)
    return a, b


def mas_hash_scalar(x: int, a: int, b: int, out_bits: int, word_bits: int = 64) -> int:
    """Multiply-add-shift: ``((a x + b) mod 2^w) >> (w - l)`` with ``l =
    out_bits`` (0 bits -> 0).  ``word_bits`` is a parameter only so tests can
    check the construction exhaustively at small widths."""
    if out_bits == 0:
        return 0
    m = (1 << word_bits) - 1
    return (((a * x) + b) & m) >> (word_bits - out_bits)


def side_hash(x: np.ndarray, seed: int, out_bits: int) -> np.ndarray:
    """``h(x)`` for an array of nonnegative indices, 64-bit words (numpy
    uint64 arithmetic wraps modulo 2^64)."""
    x = np.asarray(x, dtype=np.int64).astype(np.uint64)
    if out_bits == 0:
        return np.zeros(x.shape, dtype=np.int64)
    a, b = hash_params(seed)
    with np.errstate(over="ignore"):
        v = x * np.uint64(a) + np.uint64(b)
    return (v >> np.uint64(64 - out_bits)).astype(np.int64)


def log2_exact(P: int) -> int:
    if P < 1 or (P & (P - 1)):
        raise ValueError("P must be a power of two >= 1")
    return P.bit_length() - 1


def partition_of(i, j, P: int, seed_a: int, seed_b: int) -> np.ndarray:
    """``h(i,j) = (h_a(i) + h_b(j)) mod P`` (Lemma 1 proof)."""
    lg = log2_exact(P)
    return (side_hash(i, seed_a, lg) + side_hash(j, seed_b, lg)) % P


# ---------------------------------------------------------------------------
# Count-Sketch (Preliminaries, "Frequent items mining algorithms"; Figure 1)
# ---------------------------------------------------------------------------

def sign_params(seed: int) -> tuple[int, int]:
    """Multiplier and addend of one side's sign hash: the third and fourth
    SplitMix64 outputs of the side's seed (the first two belong to its
    partition hash)."""
    out = splitmix64(seed, 4)
    return out[2], out[3]


def side_sign(x, seed: int) -> np.ndarray:
    """``s(x)``: +1 when the top bit of ``(c x + d) mod 2^64`` is 0, else -1
    (multiply-add-shift to one bit)."""
    x = np.asarray(x, dtype=np.int64).astype(np.uint64)
    c, d = sign_params(seed)
    with np.errstate(over="ignore"):
        v = x * np.uint64(c) + np.uint64(d)
    return 1 - 2 * (v >> np.uint64(63)).astype(np.int64)


def sign_of(i, j, seed_a: int, seed_b: int) -> np.ndarray:
    """``s(i, j) = s_a(i) s_b(j)``."""
    return side_sign(i, seed_a) * side_sign(j, seed_b)


def count_sketch_terms(A: "Compressed", B: "Compressed", P: int, seed_a: int, seed_b: int,
                       mode: int = FULL) -> np.ndarray:
    """Figure 1 as written: for every outer product, every term e adds
    ``e s(e)`` to ``CS[h(e)]``.  One estimator per partition; fp64 (integer
    weights stay exact)."""
    cs = np.zeros(P)
    _, i, j, w = outer_product_terms(A, B, 0, A.n_major, mode)
    for a, b, v in zip(i.tolist(), j.tolist(), w.tolist()):
        p = int(partition_of(np.array([a]), np.array([b]), P, seed_a, seed_b)[0])
        cs[p] += v * int(sign_of(np.array([a]), np.array([b]), seed_a, seed_b)[0])
    return cs


def count_sketch(prod: "Product", P: int, seed_a: int, seed_b: int) -> np.ndarray:
    """The same from the entries: the terms of one entry add up to its weight,
    so ``CS[p]`` is the sum of ``w_e s(e)`` over the entries e in partition p."""
    p = partition_of(prod.i, prod.j, P, seed_a, seed_b)
    s = sign_of(prod.i, prod.j, seed_a, seed_b)
    cs = np.zeros(P)
    np.add.at(cs, p, prod.w * s)
    return cs


def sketch_estimate(cs: np.ndarray, i, j, P: int, seed_a: int, seed_b: int) -> np.ndarray:
    """The Count-Sketch estimate of entries (i, j): ``CS[h(e)] s(e)``."""
    return cs[partition_of(i, j, P, seed_a, seed_b)] * sign_of(i, j, seed_a, seed_b)


def count_sketch_spectrum(A: "Compressed", B: "Compressed", P: int, seed_a: int, seed_b: int,
                          freqs) -> np.ndarray:
    """``sum_p CS[p] exp(2 pi i f p / P)`` for each f of ``freqs``, from the
    inputs alone (FULL mode).  Because ``h(i,j) = (h_a(i) + h_b(j)) mod P``
    and ``s(i,j) = s_a(i) s_b(j)``, the transform of the sketch factors per
    outer product k: ``sum_k (sum_{i in a_k} a_k(i) s_a(i) w^{h_a(i)})
    (sum_{j in b_k} b_k(j) s_b(j) w^{h_b(j)})`` with ``w = exp(2 pi i f /
    P)``.  Linear in nnz per frequency, so it checks a sketch of any size."""
    lg = log2_exact(P)
    out = np.zeros(len(freqs), dtype=np.complex128)
    K = A.n_major
    # per index x of each side: s(x) and h(x)
    tabs = []
    for X, seed in ((A, seed_a), (B, seed_b)):
        x = np.arange(X.n_minor, dtype=np.int64)
        tabs.append((side_sign(x, seed).astype(np.float64), side_hash(x, seed, lg)))
    step = 1 << 20
    for n, f in enumerate(freqs):
        # s(x) w^{h(x)} for every index of each side
        g = [sg * np.exp(2j * np.pi * ((f * hx) % P) / P) for sg, hx in tabs]
        for k0 in range(0, K, step):
            k1 = min(K, k0 + step)
            per = []
            for X, gx in ((A, g[0]), (B, g[1])):
                lo, hi = int(X.ptr[k0]), int(X.ptr[k1])
                z = gx[X.idx[lo:hi]]
                if X.val is not None:
                    z = z * X.val[lo:hi].astype(np.float64)
                seg = (X.ptr[k0:k1] - lo).astype(np.int64)
                m = hi - lo
                s = np.zeros(len(seg), dtype=np.complex128)
                nz = seg < m
                if m:
                    s[nz] = np.add.reduceat(z, seg[nz])
                    # reduceat of an empty vector returns the next element: zero those
                    s[np.diff(np.append(seg, m)) == 0] = 0
                per.append(s)
            out[n] += np.sum(per[0] * per[1])
    return out


def sketch_median(estimates) -> np.ndarray:
    """The median of t instances' estimates (rows: instances)."""
    return np.median(np.asarray(estimates, dtype=np.float64), axis=0)


# ---------------------------------------------------------------------------
# Sparse inputs
# ---------------------------------------------------------------------------

@dataclass
class Compressed:
    """Compressed sparse vectors: vector k holds indices idx[ptr[k]:ptr[k+1]]
    with values val[...] (None = all ones, a {0,1} matrix)."""
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray | None
    n_minor: int

    @staticmethod
    def of(obj) -> "Compressed":
        return Compressed(np.asarray(obj.ptr, dtype=np.int64), np.asarray(obj.idx, np.int32),
                          None if obj.val is None else np.asarray(obj.val, np.float32),
                          int(obj.n_minor))

    @property
    def n_major(self) -> int:
        return len(self.ptr) - 1

    def vector(self, k: int):
        s, e = int(self.ptr[k]), int(self.ptr[k + 1])
        v = np.ones(e - s) if self.val is None else self.val[s:e].astype(np.float64)
        return self.idx[s:e].astype(np.int64), v


def total_terms(A: Compressed, B: Compressed) -> int:
    """``sum_k |a_k| |b_k|``: the number of nonzero terms over all outer
    products (Section 6, Table 2 counts these as "# of pairs")."""
    la = np.diff(A.ptr)
    lb = np.diff(B.ptr)
    return int(np.dot(la.astype(np.int64), lb.astype(np.int64)))


def dense(X: Compressed, n_major: int | None = None) -> np.ndarray:
    """Dense (n_major x n_minor) fp64 array of a compressed matrix."""
    n_major = X.n_major if n_major is None else n_major
    D = np.zeros((n_major, X.n_minor))
    for k in range(X.n_major):
        ii, vv = X.vector(k)
        D[k, ii] += vv
    return D


# ---------------------------------------------------------------------------
# Column-row product (Preliminaries, Notation)
# ---------------------------------------------------------------------------

def outer_product_terms(A: Compressed, B: Compressed, k0: int, k1: int, mode: int = FULL):
    """All nonzero terms ``a_k(i) b_k(j)`` of the outer products k in [k0, k1),
    in stream order: k ascending, then the order of a_k, then the order of b_k
    (i ascending, j ascending for sorted inputs).

    A holds the columns a_k (compressed by k, indices i), B the rows b_k
    (compressed by k, indices j).  Returns (k, i, j, w) arrays; w is the fp64
    product of the two fp32 values (exact: 24+24 mantissa bits fit in 53)."""
    la = np.diff(A.ptr[k0:k1 + 1])
    lb = np.diff(B.ptr[k0:k1 + 1])
    nt = la * lb
    T = int(nt.sum())
    ks = np.repeat(np.arange(k0, k1, dtype=np.int64), nt)
    start = np.cumsum(nt) - nt
    t = np.arange(T, dtype=np.int64) - np.repeat(start, nt)
    lbk = np.repeat(lb, nt)
    ia = A.ptr[ks] + t // np.maximum(lbk, 1)
    jb = B.ptr[ks] + t % np.maximum(lbk, 1)
    i = A.idx[ia].astype(np.int64)
    j = B.idx[jb].astype(np.int64)
    if A.val is None and B.val is None:
        w = np.ones(T)
    else:
        wa = np.ones(T) if A.val is None else A.val[ia].astype(np.float64)
        wb = np.ones(T) if B.val is None else B.val[jb].astype(np.float64)
        w = wa * wb
    if mode == UPPER:
        keep = i < j
        ks, i, j, w = ks[keep], i[keep], j[keep], w[keep]
    return ks, i, j, w


def exact_product_loop(A: Compressed, B: Compressed, mode: int = FULL) -> dict:
    """The definition written as loops: for each k, for each i in a_k, for
    each j in b_k, ``C[(i, j)] += a_k(i) b_k(j)``.  For tiny inputs only."""
    C: dict = {}
    for k in range(A.n_major):
        ii, va = A.vector(k)
        jj, vb = B.vector(k)
        for x in range(len(ii)):
            for y in range(len(jj)):
                i, j = int(ii[x]), int(jj[y])
                if mode == UPPER and not i < j:
                    continue
                C[(i, j)] = C.get((i, j), 0.0) + float(va[x]) * float(vb[y])
    return C


@dataclass
class Product:
    """Nonzero entries of C sorted by (i, j): arrays i, j, w (fp64; counts are
    exact integers in fp64 up to 2^53) and the number of terms processed."""
    i: np.ndarray
    j: np.ndarray
    w: np.ndarray
    terms: int
    n_cols: int

    def keys(self) -> np.ndarray:
        return self.i * self.n_cols + self.j

    def as_dict(self) -> dict:
        return {(int(a), int(b)): float(c) for a, b, c in zip(self.i, self.j, self.w)}


def _reduce(keys: np.ndarray, w: np.ndarray):
    uk, inv = np.unique(keys, return_inverse=True)
    return uk, np.bincount(inv, weights=w, minlength=len(uk))


def exact_product(A: Compressed, B: Compressed, mode: int = FULL,
                  chunk_terms: int = 20_000_000) -> Product:
    """C = sum_k a_k b_k exactly: every term of every outer product is added
    into its entry.  Terms are generated a range of k at a time; equal keys
    are summed with a sort (np.unique) and a bincount."""
    n_cols = B.n_minor
    la = np.diff(A.ptr)
    lb = np.diff(B.ptr)
    nt = np.cumsum(la.astype(np.int64) * lb.astype(np.int64))
    K = A.n_major
    parts_k, parts_w = [], []
    terms = 0
    k0 = 0
    while k0 < K:
        base = nt[k0 - 1] if k0 else 0
        k1 = int(np.searchsorted(nt, base + chunk_terms, side="right"))
        k1 = max(k1, k0 + 1)
        k1 = min(k1, K)
        _, i, j, w = outer_product_terms(A, B, k0, k1, mode)
        terms += len(i)
        uk, uw = _reduce(i * n_cols + j, w)
        parts_k.append(uk)
        parts_w.append(uw)
        k0 = k1
    if parts_k:
        uk, uw = _reduce(np.concatenate(parts_k), np.concatenate(parts_w))
    else:
        uk, uw = np.zeros(0, np.int64), np.zeros(0)
    return Product(uk // n_cols, uk % n_cols, uw, terms, n_cols)


def split_by_partition(prod: Product, P: int, seed_a: int, seed_b: int) -> list[Product]:
    """Per-partition tables: entry (i, j) goes to partition h(i, j) and to no
    other (Lemma 1; Section 4 "Our approach")."""
    p = partition_of(prod.i, prod.j, P, seed_a, seed_b)
    out = []
    for q in range(P):
        m = p == q
        out.append(Product(prod.i[m], prod.j[m], prod.w[m], -1, prod.n_cols))
    return out


def partition_entries(A: Compressed, B: Compressed, P: int, p: int, seed_a: int, seed_b: int,
                      chunk: int = 1_000_000) -> Product:
    """All entries of partition p, exactly, without the rest of the product
    (FULL mode, {0,1} or real values).  A term a_k(i) b_k(j) lands in p when
    ``h_b(j) = (p - h_a(i)) mod P`` (Lemma 1: the partition of a pair is fixed
    by its two side hashes).  So for each outer product, every entry i of a_k
    is joined with the entries j of b_k whose side hash equals its target:
    the (k, h_b(j)) pairs of B are sorted once per chunk of outer products and
    each (k, target) is looked up; equal (i, j) are then summed."""
    lg = log2_exact(P)
    n_cols = B.n_minor
    keys_all, w_all = [], []
    for k0 in range(0, A.n_major, chunk):
        k1 = min(A.n_major, k0 + chunk)
        a_lo, a_hi = int(A.ptr[k0]), int(A.ptr[k1])
        b_lo, b_hi = int(B.ptr[k0]), int(B.ptr[k1])
        ka = np.repeat(np.arange(k0, k1, dtype=np.int64), np.diff(A.ptr[k0:k1 + 1]))
        kb = np.repeat(np.arange(k0, k1, dtype=np.int64), np.diff(B.ptr[k0:k1 + 1]))
        ia = A.idx[a_lo:a_hi].astype(np.int64)
        jb = B.idx[b_lo:b_hi].astype(np.int64)
        va = np.ones(len(ia)) if A.val is None else A.val[a_lo:a_hi].astype(np.float64)
        vb = np.ones(len(jb)) if B.val is None else B.val[b_lo:b_hi].astype(np.float64)
        target = (p - side_hash(ia, seed_a, lg)) % P
        bkey = kb * P + side_hash(jb, seed_b, lg)
        order = np.argsort(bkey, kind="stable")
        bkey, jb, vb = bkey[order], jb[order], vb[order]
        akey = ka * P + target
        lo = np.searchsorted(bkey, akey, side="left")
        hi = np.searchsorted(bkey, akey, side="right")
        cnt = hi - lo
        rep = np.repeat(np.arange(len(ia)), cnt)
        off = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        pos = np.repeat(lo, cnt) + off
        keys_all.append(ia[rep] * n_cols + jb[pos])
        w_all.append(va[rep] * vb[pos])
    if keys_all:
        uk, uw = _reduce(np.concatenate(keys_all), np.concatenate(w_all))
    else:
        uk, uw = np.zeros(0, np.int64), np.zeros(0)
    return Product(uk // n_cols, uk % n_cols, uw, -1, n_cols)


def partition_term_counts(A: Compressed, B: Compressed, P: int, seed_a: int, seed_b: int,
                          mode: int = FULL, chunk_terms: int = 20_000_000) -> np.ndarray:
    """Number of terms (not entries) of all outer products landing in each
    partition: the per-processor work of Theorem 1 / Table 4."""
    la = np.diff(A.ptr)
    lb = np.diff(B.ptr)
    nt = np.cumsum(la.astype(np.int64) * lb.astype(np.int64))
    out = np.zeros(P, dtype=np.int64)
    K = A.n_major
    k0 = 0
    while k0 < K:
        base = nt[k0 - 1] if k0 else 0
        k1 = min(max(int(np.searchsorted(nt, base + chunk_terms, side="right")), k0 + 1), K)
        _, i, j, _ = outer_product_terms(A, B, k0, k1, mode)
        out += np.bincount(partition_of(i, j, P, seed_a, seed_b), minlength=P)
        k0 = k1
    return out


def interval_terms(a_idx, a_val, b_idx, b_val, q: int, r: int, P: int, seed_a: int,
                   seed_b: int):
    """``E_L^{ab}`` for ``L = [q, r)`` (Lemma 1): the entries of the single
    outer product ``ab`` whose hash lies in [q, r), found by testing every
    pair.  Returns a list of (i, j, w) in (a order, b order)."""
    out = []
    for x in range(len(a_idx)):
        for y in range(len(b_idx)):
            i, j = int(a_idx[x]), int(b_idx[y])
            h = int(partition_of(np.array([i]), np.array([j]), P, seed_a, seed_b)[0])
            if q <= h < r:
                out.append((i, j, float(a_val[x]) * float(b_val[y])))
    return out


def entry(A_rows: Compressed, B_cols: Compressed, i: int, j: int) -> float:
    """One entry by its definition as an inner product: row i of A (compressed
    by i, indices k) times column j of B (compressed by j, indices k)."""
    ka, va = A_rows.vector(i)
    kb, vb = B_cols.vector(j)
    common, xa, xb = np.intersect1d(ka, kb, assume_unique=True, return_indices=True)
    return float(np.dot(va[xa], vb[xb]))


# ---------------------------------------------------------------------------
# Heaviest entries (Section 6)
# ---------------------------------------------------------------------------

def topk(i: np.ndarray, j: np.ndarray, w: np.ndarray, k: int, upper_only: bool = False):
    """The k heaviest entries ordered by weight descending, then i, then j
    ascending.  ``upper_only`` keeps pairs i < j only."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    w = np.asarray(w, np.float64)
    if upper_only:
        m = i < j
        i, j, w = i[m], j[m], w[m]
    order = np.lexsort((j, i, -np.abs(w)))[:k]
    return i[order], j[order], w[order]


def certified_topk_pairs(T: Compressed, k: int, n_hot: int = 2048, chunk: int = 2_000_000):
    """The k heaviest pairs i < j of ``T^T T`` for a {0,1} matrix T (rows =
    transactions), exactly, without the whole product.  Every entry satisfies
    ``C(i,j) <= min(C(i,i), C(j,j))`` (a pair occurs only in transactions that
    hold both items), so once the pairs among the n_hot most frequent items are
    counted exactly (``H^T H`` with H the columns of those items, a sparse
    matrix product, summed over chunks of transactions), any pair with an item
    outside that set weighs at most the largest support outside it.  If the
    k-th heaviest counted pair is heavier than that bound, the counted pairs'
    top k (weight descending, then i, then j) is the product's top k;
    otherwise n_hot doubles.  Returns (i, j, w, certificate dict)."""
    import scipy.sparse as sp
    deg = prefix_item_counts(T)
    n = T.n_minor
    while True:
        h = min(n_hot, n)
        hot = top_items(deg, h)
        rank = np.full(n, -1, dtype=np.int64)
        rank[hot] = np.arange(h)
        C = np.zeros((h, h), dtype=np.int64)
        K = T.n_major
        for k0 in range(0, K, chunk):
            k1 = min(K, k0 + chunk)
            lo, hi = int(T.ptr[k0]), int(T.ptr[k1])
            idx = T.idx[lo:hi].astype(np.int64)
            row = np.repeat(np.arange(k1 - k0), np.diff(T.ptr[k0:k1 + 1]))
            r = rank[idx]
            m = r >= 0
            H = sp.csr_matrix((np.ones(int(m.sum()), dtype=np.int64), (row[m], r[m])),
                              shape=(k1 - k0, h))
            C += (H.T @ H).toarray()
        a, b = np.triu_indices(h, k=1)
        i, j = hot[a], hot[b]
        sw = np.where(i < j, 0, 1)          # order each pair as i < j
        i, j = np.where(sw == 0, i, j), np.where(sw == 0, j, i)
        w = C[a, b].astype(np.float64)
        ti, tj, tw = topk(i, j, w, k)
        outside = np.ones(n, dtype=bool)
        outside[hot] = False
        bound = float(deg[outside].max()) if outside.any() else 0.0
        if len(tw) == k and tw[-1] > bound:
            return ti, tj, tw, dict(n_hot=h, bound=bound, kth=float(tw[-1]))
        if h >= n:
            return ti, tj, tw, dict(n_hot=h, bound=bound, kth=float(tw[-1]) if len(tw) else 0.0)
        n_hot *= 2


# ---------------------------------------------------------------------------
# Space-Saving (Preliminaries)
# ---------------------------------------------------------------------------

def space_saving(stream, ell: int) -> dict:
    """Weighted Space-Saving over a stream of (key, w), w > 0, with ``ell``
    counters.  Returns {key: (count, overestimation)}; the upper bound on the
    key's weight is ``count`` and the lower bound ``count - overestimation``.

    * key already recorded: count += w;
    * a free counter: record (key, w, 0);
    * otherwise the counter of minimum count (ties: smallest key) is given to
      the key as (key, min + w, min).
    A lazy heap of (count, key) finds the minimum."""
    summ: dict = {}
    heap: list = []
    for key, w in stream:
        if key in summ:
            c, o = summ[key]
            summ[key] = (c + w, o)
            heapq.heappush(heap, (c + w, key))
        elif len(summ) < ell:
            summ[key] = (w, 0)
            heapq.heappush(heap, (w, key))
        else:
            while True:
                c, victim = heapq.heappop(heap)
                if victim in summ and summ[victim][0] == c:
                    break
            del summ[victim]
            summ[key] = (c + w, c)
            heapq.heappush(heap, (c + w, key))
    return summ


def partition_streams(A: Compressed, B: Compressed, P: int, seed_a: int, seed_b: int,
                      mode: int = FULL):
    """Per-partition term streams in stream order (k ascending, then i, then
    j): the input each Space-Saving summary of the CRoP algorithm sees
    (Figure 1: entries of each outer product go to the summary of their
    bucket)."""
    ks, i, j, w = outer_product_terms(A, B, 0, A.n_major, mode)
    order = np.lexsort((j, i, ks))
    ks, i, j, w = ks[order], i[order], j[order], w[order]
    p = partition_of(i, j, P, seed_a, seed_b)
    n_cols = B.n_minor
    out = []
    for q in range(P):
        m = p == q
        out.append(list(zip((i[m] * n_cols + j[m]).tolist(), w[m].tolist())))
    return out


def bucket_summaries(A: Compressed, B: Compressed, P: int, ell: int, seed_a: int, seed_b: int,
                     mode: int = FULL):
    """Figure 1 with one Space-Saving summary of ``ell`` counters per bucket
    (the paper's regime of many buckets): every partition's stream, in stream
    order, through :func:`space_saving`.  The streams are grouped with one
    stable sort by partition rather than one scan per partition, so many
    buckets stay affordable.  Returns (p, key, count, overestimation) arrays
    over every recorded key, key = i * n_cols + j."""
    ks, i, j, w = outer_product_terms(A, B, 0, A.n_major, mode)
    order = np.lexsort((j, i, ks))
    i, j, w = i[order], j[order], w[order]
    p = partition_of(i, j, P, seed_a, seed_b)
    grp = np.argsort(p, kind="stable")
    p, key, w = p[grp], (i * B.n_minor + j)[grp], w[grp]
    cuts = np.flatnonzero(np.diff(p)) + 1
    P_out, K_out, C_out, O_out = [], [], [], []
    for lo, hi in zip(np.concatenate([[0], cuts]), np.concatenate([cuts, [len(p)]])):
        if lo == hi:
            continue
        summ = space_saving(zip(key[lo:hi].tolist(), w[lo:hi].tolist()), ell)
        for k, (c, o) in summ.items():
            P_out.append(int(p[lo]))
            K_out.append(k)
            C_out.append(c)
            O_out.append(o)
    return (np.array(P_out, np.int64), np.array(K_out, np.int64), np.array(C_out, np.float64),
            np.array(O_out, np.float64))


# ---------------------------------------------------------------------------
# Heavy-pair predictor (a 2 -> 64 -> 64 -> 1 MLP; not in the paper)
# ---------------------------------------------------------------------------
# Parameter vector layout (fp32 master weights), shared with the CUDA kernels
# only through this documented layout: W1[64][2], b1[64], W2[64][64], b2[64],
# w3[64], b3[1].
MLP_H = 64
MLP_SIZES = (("W1", (64, 2)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("w3", (64,)),
             ("b3", (1,)))
MLP_NPARAM = sum(int(np.prod(s)) for _, s in MLP_SIZES)


def mlp_unpack(theta):
    out, o = {}, 0
    for name, shape in MLP_SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def mlp_pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in MLP_SIZES])


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(theta, X, rounding: bool = True):
    """y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 per row of X (M x 2).
    With ``rounding`` the operands of the two matrix products (x, W1, the
    first hidden layer, W2) are bf16, as the tensor-core kernels use them;
    everything else is fp64."""
    p = mlp_unpack(theta)
    rd = bf16_round if rounding else (lambda a: np.asarray(a, np.float64))
    Xb = rd(X)
    W1b = rd(p["W1"])
    Z1 = Xb @ W1b.T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    H1b = rd(H1)
    W2b = rd(p["W2"])
    Z2 = H1b @ W2b.T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, dict(Xb=Xb, W1b=W1b, Z1=Z1, H1b=H1b, W2b=W2b, Z2=Z2, H2=H2, p=p)


def mlp_loss_grad(theta, X, t, rounding: bool = True, n_total: int | None = None):
    """Mean squared error L = sum((y - t)^2) / n_total and its gradient with
    respect to the master parameters (straight through the bf16 copies).  With
    ``rounding`` the backward products use bf16 operands (dZ2, dZ1, the
    saved activations) like the kernels do; the bias gradients of the hidden
    layers are the sums over the batch of those same bf16 dZ2 and dZ1 (the
    kernels form them as products with a row of ones)."""
    y, c = mlp_forward(theta, X, rounding)
    rd = bf16_round if rounding else (lambda a: np.asarray(a, np.float64))
    n = len(y) if n_total is None else n_total
    r = y - t
    L = float(np.dot(r, r) / n)
    dy = 2.0 * r / n
    p = c["p"]
    dw3 = c["H2"].T @ dy
    db3 = np.array([dy.sum()])
    dZ2 = np.outer(dy, p["w3"]) * (c["Z2"] > 0)
    dZ2b = rd(dZ2)
    db2 = dZ2b.sum(axis=0)
    dW2 = dZ2b.T @ c["H1b"]
    dH1 = dZ2b @ c["W2b"]
    dZ1 = dH1 * (c["Z1"] > 0)
    dZ1b = rd(dZ1)
    db1 = dZ1b.sum(axis=0)
    dW1 = dZ1b.T @ c["Xb"]
    g = mlp_pack(dict(W1=dW1, b1=db1, W2=dW2, b2=db2, w3=dw3, b3=db3))
    return L, g, y


def mlp_init(seed: int) -> np.ndarray:
    """He-style initial parameters (fp32 values)."""
    rng = np.random.default_rng(seed)
    d = dict(W1=rng.normal(0, np.sqrt(2 / 2), (64, 2)), b1=np.full(64, 0.01),
             W2=rng.normal(0, np.sqrt(2 / 64), (64, 64)), b2=np.full(64, 0.01),
             w3=rng.normal(0, np.sqrt(1 / 64), 64), b3=np.zeros(1))
    return mlp_pack(d).astype(np.float32).astype(np.float64)


def adam_step(theta, m, v, g, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of fp32 master parameters."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def marginal_features(counts_i, counts_j, scale):
    """Predictor inputs of a pair: log(1 + c_i) / scale, log(1 + c_j) / scale,
    the items' counts in a prefix of the stream."""
    return np.stack([np.log1p(counts_i) / scale, np.log1p(counts_j) / scale], axis=1)


def prefix_item_counts(prefix: Compressed) -> np.ndarray:
    """c_x: how many vectors (transactions) of the prefix hold item x."""
    return np.bincount(prefix.idx.astype(np.int64), minlength=prefix.n_minor).astype(np.int64)


def top_items(counts: np.ndarray, R: int) -> np.ndarray:
    """The R items of largest count, by count descending, ties by the smaller
    item id (a reading: which of several items tied at the R-th count is
    taken is not fixed by anything)."""
    order = np.lexsort((np.arange(len(counts)), -np.asarray(counts)))
    return order[:R]


def candidate_pairs(prefix: Compressed, R: int):
    """Candidate heavy pairs from a prefix of the stream: every pair i < j of
    the R items of largest prefix count, sorted by (i, j), with features
    (log(1 + c_i), log(1 + c_j)) / log(1 + max c).  Returns (i, j, X, c)."""
    c = prefix_item_counts(prefix)
    items = np.sort(top_items(c, R))
    a, b = np.triu_indices(len(items), k=1)
    i, j = items[a], items[b]
    scale = np.log1p(c.max()) if len(c) else 0.0
    X = marginal_features(c[i], c[j], scale) if scale > 0 else np.zeros((len(i), 2))
    return i, j, X, c
