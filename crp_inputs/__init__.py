"""Seeded synthetic inputs for the column-row product workloads.

This module only produces input matrices (as numpy arrays).  It holds none of
the product's arithmetic: no hashing, partitioning or accumulation.  The CUDA
path and the CPU oracle both consume what it returns, and neither imports the
other.

The generator itself is C (``gen.c``, Philox4x32-10 counter-based streams,
OpenMP across transactions), compiled on first use with the host ``gcc``.

Workloads (all seeded, all synthetic) stand in for the datasets of the paper's
case study (Section 6, Table 2: FIMI / UCI transaction and bag-of-words data),
which are not available here:

* ``c1``  20,000 transactions x 1,000 items, lengths Poisson(10) clamped to
  [2, 40], items Zipf(1.1)                              (co-occurrence, T^T T)
* ``c2``  10M transactions x 100,000 items, Poisson(20) clamped to [2, 100],
  Zipf(1.0)                                            (co-occurrence, T^T T)
* ``c3``  100,000 x 100,000 column-stochastic A, column nnz power law with
  exponent 2.1 on [5, 2000], lognormal(0,1) values normalised per column
  (real product A A)
* ``c4``  50M transactions x 1M items, Poisson(15), Zipf(1.2)  (heavy entries)
* ``c5``  4,096 problems: transactions log-uniform [100, 2e5], items
  log-uniform [1e3, 1e5], Zipf exponent U[0.8, 1.3], Poisson(12) lengths
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "_crp_gen.so")
_lock = threading.Lock()
_lib = None

#: data seed of workload c<N> is 1000 + N
DATA_SEED_BASE = 1000


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into ``_crp_gen.so`` (gcc, OpenMP, no FP contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            f32p = ctypes.POINTER(ctypes.c_float)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.crp_gen_tx_lengths.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                               i64p]
            lib.crp_gen_tx_items.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_double, i64p, i32p]
            lib.crp_gen_powerlaw_counts.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                                    ctypes.c_double, ctypes.c_int32,
                                                    ctypes.c_int32, i64p]
            lib.crp_gen_stochastic_cols.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                                    ctypes.c_int32, ctypes.c_double,
                                                    ctypes.c_double, i64p, i32p, f32p]
            lib.crp_gen_transpose.argtypes = [ctypes.c_int64, ctypes.c_int32, i64p, i32p, f32p,
                                              i64p, i32p, f32p]
            lib.crp_gen_philox_block.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 4 + [u32p]
            lib.crp_gen_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_int32]
            lib.crp_gen_uniform.restype = ctypes.c_double
            for f in (lib.crp_gen_tx_lengths, lib.crp_gen_tx_items, lib.crp_gen_powerlaw_counts,
                      lib.crp_gen_stochastic_cols, lib.crp_gen_transpose):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


@dataclass
class Sparse:
    """A compressed sparse matrix: ``ptr`` (int64, n_major+1), ``idx`` (int32),
    ``val`` (float32 or None for a {0,1} matrix), minor dimension ``n_minor``."""
    ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray | None
    n_minor: int

    @property
    def n_major(self) -> int:
        return int(self.ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.ptr[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.ptr)


def philox_block(seed: int, ctr: tuple[int, int, int, int]) -> tuple[int, int, int, int]:
    """One raw Philox4x32-10 output block (key = seed low/high words)."""
    out = np.zeros(4, dtype=np.uint32)
    _load().crp_gen_philox_block(seed, *[c & 0xFFFFFFFF for c in ctr], _p(out, ctypes.c_uint32))
    return tuple(int(x) for x in out)


def transactions(seed: int, m: int, n: int, lam: float, lmin: int, lmax: int,
                 zipf_s: float) -> Sparse:
    """A {0,1} transaction matrix T (CSR, rows = transactions, sorted distinct
    item ids per row).  Row lengths ~ Poisson(lam) clamped to [lmin, lmax]
    (``lmax < lmin`` = no clamp), items Zipf(zipf_s) over [n]."""
    lib = _load()
    lens = np.empty(m, dtype=np.int64)
    if m:
        rc = lib.crp_gen_tx_lengths(seed, m, n, lam, lmin, lmax, _p(lens, ctypes.c_int64))
        assert rc == 0
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=ptr[1:])
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    if m:
        rc = lib.crp_gen_tx_items(seed, m, n, zipf_s, _p(ptr, ctypes.c_int64),
                                  _p(idx, ctypes.c_int32))
        assert rc == 0, "generator allocation failed"
    return Sparse(ptr, idx, None, n)


def stochastic(seed: int, n: int, alpha: float = 2.1, cmin: int = 5, cmax: int = 2000,
               mu: float = 0.0, sigma: float = 1.0) -> Sparse:
    """Column-stochastic n x n matrix A in CSC (columns sum to 1)."""
    lib = _load()
    cnt = np.empty(n, dtype=np.int64)
    lib.crp_gen_powerlaw_counts(seed, n, alpha, cmin, min(cmax, n), _p(cnt, ctypes.c_int64))
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=ptr[1:])
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    val = np.empty(int(ptr[-1]), dtype=np.float32)
    rc = lib.crp_gen_stochastic_cols(seed, n, n, mu, sigma, _p(ptr, ctypes.c_int64),
                                     _p(idx, ctypes.c_int32), _p(val, ctypes.c_float))
    assert rc == 0
    return Sparse(ptr, idx, val, n)


def transpose(s: Sparse) -> Sparse:
    """The same matrix compressed along the other dimension."""
    lib = _load()
    tptr = np.zeros(s.n_minor + 1, dtype=np.int64)
    tidx = np.empty(s.nnz, dtype=np.int32)
    tval = np.empty(s.nnz, dtype=np.float32) if s.val is not None else None
    rc = lib.crp_gen_transpose(s.n_major, s.n_minor, _p(s.ptr, ctypes.c_int64),
                               _p(s.idx, ctypes.c_int32), _p(s.val, ctypes.c_float),
                               _p(tptr, ctypes.c_int64), _p(tidx, ctypes.c_int32),
                               _p(tval, ctypes.c_float))
    assert rc == 0
    return Sparse(tptr, tidx, tval, s.n_major)


def uniform(seed: int, stream: int, item: int, which: int = 0) -> float:
    return float(_load().crp_gen_uniform(seed, stream, item, which))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class TxWorkload:
    name: str
    m: int
    n: int
    lam: float
    lmin: int
    lmax: int
    zipf_s: float
    seed: int

    def scaled(self, m: int | None = None, n: int | None = None) -> "TxWorkload":
        return TxWorkload(self.name, m if m is not None else self.m,
                          n if n is not None else self.n, self.lam, self.lmin, self.lmax,
                          self.zipf_s, self.seed)

    def generate(self) -> Sparse:
        return transactions(self.seed, self.m, self.n, self.lam, self.lmin, self.lmax,
                            self.zipf_s)


C1 = TxWorkload("c1", 20_000, 1_000, 10.0, 2, 40, 1.1, DATA_SEED_BASE + 1)
C2 = TxWorkload("c2", 10_000_000, 100_000, 20.0, 2, 100, 1.0, DATA_SEED_BASE + 2)
C4 = TxWorkload("c4", 50_000_000, 1_000_000, 15.0, 0, -1, 1.2, DATA_SEED_BASE + 4)

C3_N = 100_000
C3_SEED = DATA_SEED_BASE + 3


def c3(n: int = C3_N, cmax: int = 2000) -> tuple[Sparse, Sparse]:
    """Real workload c3: returns (CSC of A, CSR of A) for C = A A."""
    a_csc = stochastic(C3_SEED, n, 2.1, 5, cmax)
    return a_csc, transpose(a_csc)


C5_SEED = DATA_SEED_BASE + 5


def c5_params(nprob: int = 4096, m_range=(100, 200_000), n_range=(1_000, 100_000),
              s_range=(0.8, 1.3), lam: float = 12.0) -> list[TxWorkload]:
    """Per-problem shapes of the batched workload c5 (log-uniform sizes)."""
    out = []
    for p in range(nprob):
        u0, u1, u2 = (uniform(C5_SEED, 7, p, w) for w in range(3))
        m = int(round(math.exp(math.log(m_range[0]) + u0 * (math.log(m_range[1]) -
                                                             math.log(m_range[0])))))
        n = int(round(math.exp(math.log(n_range[0]) + u1 * (math.log(n_range[1]) -
                                                             math.log(n_range[0])))))
        s = s_range[0] + u2 * (s_range[1] - s_range[0])
        out.append(TxWorkload(f"c5[{p}]", m, n, lam, 0, -1, s, C5_SEED * 100_003 + p))
    return out


# Fixed hash seeds of the recorded workloads (h_a and h_b must differ).
SEED_A = 0x243F6A8885A308D3
SEED_B = 0x13198A2E03707344
