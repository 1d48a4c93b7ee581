"""Write the oracle's heaviest pairs of the full-size co-occurrence workloads.

Calls only the oracle (and the seeded input generators): for the
10M-transaction workload (100,000 items, Poisson(20) in [2,100], Zipf(1.0))
and the 50M-transaction heavy-entry workload (1M items, Poisson(15),
Zipf(1.2)), the k heaviest pairs i < j of T^T T, each certified exact by the
support bound (oracle.crp_oracle.certified_topk_pairs; Section 6 reports the
heaviest pairs of the case study).  The GPU benchmark and the full-size GPU
tests judge the library's top-k against these files.  Each file records the
SHA-256 of the input arrays it was computed from, so a reader can check that
it generated the same input.

    python tests/golden/make_topk_fixtures.py [c2] [c4]
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import crp_inputs as ci  # noqa: E402
from oracle import crp_oracle as O  # noqa: E402

JOBS = {"c2": (ci.C2, 2000, 2048), "c4": (ci.C4, 16384, 4096)}


def input_digest(T) -> str:
    h = hashlib.sha256()
    h.update(T.ptr.tobytes())
    h.update(T.idx.tobytes())
    return h.hexdigest()


def main(names):
    for name in names:
        w, k, n_hot = JOBS[name]
        t0 = time.time()
        T = w.generate()
        digest = input_digest(T)
        i, j, wt, cert = O.certified_topk_pairs(O.Compressed.of(T), k, n_hot)
        path = os.path.join(HERE, f"{name}_top{k}.txt")
        with open(path, "w") as f:
            f.write(f"# The {k} heaviest pairs i < j of T^T T (weight descending, then i, j),\n"
                    f"# exact: written by tests/golden/make_topk_fixtures.py from the oracle\n"
                    f"# (certified_topk_pairs; Section 6, heaviest pairs of the case study).\n"
                    f"# workload {w.name}: {w.m} transactions x {w.n} items, Poisson({w.lam:g})"
                    f" clamp [{w.lmin},{w.lmax}], Zipf({w.zipf_s:g}), data seed {w.seed}\n"
                    f"# input sha256 {digest}\n"
                    f"# certificate: pairs among the {cert['n_hot']} most frequent items counted;"
                    f" k-th weight {cert['kth']:.0f} > largest support outside {cert['bound']:.0f}\n"
                    f"# format: i j weight\n")
            for a, b, c in zip(i.tolist(), j.tolist(), wt.tolist()):
                f.write(f"{a} {b} {int(c)}\n")
        print(f"{name}: {path} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(JOBS))
