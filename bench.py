#!/usr/bin/env python3
"""Throughput of the exact column-row co-occurrence product on GB300.

Workload (default): 10M transactions x 100,000 items, lengths Poisson(20)
clamped to [2, 100], items Zipf(1.0), seeded synthetic data; exact int32
counts of T^T T (every entry, FULL mode) in per-partition HBM hash tables,
then the 1,000 heaviest pairs (i < j).

One step = reset the partition tables, enumerate + combine + flush every
outer-product term (crp_outer_accumulate), crp_sync, and crp_topk(1000).
Prints one JSON line: the metric, the roofline of the dominant kernel, the oracle baseline, the end-to-end figure and the clocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "outer-product terms/sec on 1 GB300 (exact) and % of HBM roofline; top-k weight err"
# Algorithmic bytes per outer-product term of the update roofline: one random
# read-modify-write of a 32-byte HBM sector (the entry's slot).
BYTES_PER_TERM_UPDATE = 64.0
SLOT_BYTES = 16.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m", type=int, default=None, help="transactions (default: workload's)")
    ap.add_argument("--P", type=int, default=1024)
    ap.add_argument("--groups", type=int, default=1)
    ap.add_argument("--tile", type=int, default=64)
    ap.add_argument("--smem-slots", type=int, default=8192)
    ap.add_argument("--hot", type=int, default=0, help="hot-block items (direct/routed)")
    ap.add_argument("--warm", type=int, default=0, help="warm-stripe items (direct/routed)")
    ap.add_argument("--load", type=int, default=0, help="target table load %% (0 = library default)")
    ap.add_argument("--topk", type=int, default=1000)
    ap.add_argument("--no-match", action="store_true")
    ap.add_argument("--paper-regime", action="store_true",
                    help="c4: also run the paper's many-buckets, two-counter summary regime")
    ap.add_argument("--sketch", action="store_true",
                    help="also keep the per-partition Count-Sketch (direct mode)")
    ap.add_argument("--mode", choices=["direct", "smem", "routed"], default="direct",
                    help="accumulation variant (CRP_PLAN_DIRECT / on-chip table / CRP_PLAN_ROUTED)")
    ap.add_argument("--autotune", type=int, default=2_500_000,
                    help="outer products of the workload the autotuner samples (0 = off: use "
                         "--P/--mode/--tile/--smem-slots)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", choices=["c2", "c1", "c3", "c4", "c5"], default="c2",
                    help="c2 is the graded line; the others report the remaining workloads")
    ap.add_argument("--c5-problems", type=int, default=4096)
    ap.add_argument("--c5-mmax", type=int, default=200_000)
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("crp_accumulate.cu", "crp_route.cu", "crp_device.cuh", "crp_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1210_0461_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def oracle_top_pairs(name: str, T):
    """The oracle's certified heaviest pairs of a full-size workload, read from
    the fixture tests/golden/<name>_top<k>.txt (written by
    tests/golden/make_topk_fixtures.py, which calls only the oracle), if the
    fixture was computed from these very input arrays (SHA-256 recorded in
    it).  Returns (list of (i, j, w) in rank order, None) or (None, reason)."""
    import glob
    files = sorted(glob.glob(os.path.join(ROOT, "tests", "golden", f"{name}_top*.txt")))
    if not files:
        return None, "no oracle fixture"
    path = files[0]
    want = None
    rows = []
    for line in open(path):
        if line.startswith("# input sha256 "):
            want = line.split()[-1]
        elif line.strip() and not line.startswith("#"):
            a, b, c = line.split()
            rows.append((int(a), int(b), float(c)))
    h = hashlib.sha256()
    h.update(T.ptr.tobytes())
    h.update(T.idx.tobytes())
    if h.hexdigest() != want:
        return None, "input differs from the one the oracle fixture was computed from"
    return rows, None


def topk_weight_error(ti, tj, oracle_rows, k: int):
    """Reading of "top-k weight error": 1 - sum of the true weights of the
    returned pairs / sum of the true top-k weights, with the true weights from
    the oracle's certified list.  A returned pair outside that list weighs at
    most its last weight: the error is then an interval.  Returns a dict with
    the error (its upper end), its lower end, the pairs outside the list, and
    whether the returned list equals the oracle's top k in order."""
    look = {(a, b): c for a, b, c in oracle_rows}
    top_sum = sum(c for _, _, c in oracle_rows[:k])
    floor_w = oracle_rows[-1][2]
    known = unknown = 0.0
    n_unknown = 0
    for a, b in zip([int(x) for x in ti], [int(x) for x in tj]):
        if (a, b) in look:
            known += look[(a, b)]
        else:
            n_unknown += 1
            unknown += floor_w
    exact = (len(ti) == k and
             [(int(a), int(b)) for a, b in zip(ti, tj)] == [(a, b) for a, b, _ in oracle_rows[:k]])
    return {"topk_weight_err": 1.0 - known / top_sum,
            "topk_weight_err_low": 1.0 - (known + unknown) / top_sum,
            "pairs_outside_oracle_list": n_unknown, "equals_oracle_topk": exact,
            "judged_by": f"oracle certified top-{len(oracle_rows)} (tests/golden)"}


def workload(args):
    import crp_inputs as ci
    w = ci.C2 if args.m is None else ci.C2.scaled(m=args.m)
    return w


def cpu_baseline(T, budget_s: float, mode: int = 0):
    """The oracle, as it stands, on a bounded prefix of the workload's
    transactions (doubled until one pass takes at least 2/3 of ``budget_s``
    seconds: 10-20 s of CPU work for the default budget)."""
    from oracle import crp_oracle as O
    import numpy as np
    m = 2000
    while True:
        sub = O.Compressed(T.ptr[:m + 1], T.idx[:T.ptr[m]], None, T.n_minor)
        t0 = time.perf_counter()
        prod = O.exact_product(sub, sub, mode)
        dt = time.perf_counter() - t0
        if dt >= budget_s * 2 / 3 or m * 2 > T.n_major:
            break
        m *= 2
    return {"value": prod.terms / dt, "unit": "terms/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m} transactions ({prod.terms} terms, {len(prod.i)} entries), "
                      f"{dt:.2f} s single-threaded numpy", "seconds": dt}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores, each step a
    bounded sample of the workload."""
    import numpy as np
    from oracle import crp_oracle as O
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    T = w.generate()
    m = min(T.n_major, 40_000)
    sub = O.Compressed(T.ptr[:m + 1], T.idx[:T.ptr[m]], None, T.n_minor)
    for _ in range(args.warmup):
        O.exact_product(sub, sub, O.FULL)
    t0 = time.perf_counter()
    terms = 0
    for _ in range(args.steps):
        p = O.exact_product(sub, sub, O.FULL)
        O.topk(p.i, p.j, p.w, args.topk, upper_only=True)
        terms += p.terms
    dt = time.perf_counter() - t0
    v = terms / dt
    sample = f"first {m} transactions of {w.name} per step ({terms // max(args.steps, 1)} terms)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "terms/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i64", "data": "synthetic",
        "config": {"workload": f"{w.name} sample: {sample}"},
        "cpu_baseline": {"value": v, "unit": "terms/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "terms/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def _line(value, ms, args, dtype, config, extra=None):
    out = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    out.update(extra or {})
    print(json.dumps(out), flush=True)


def run_other(args):
    """The remaining workloads, one JSON line each (not the graded line)."""
    import numpy as np
    import torch
    import crp_inputs as ci
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.workload == "c1":
        T = ci.C1.generate()
        d = crp.to_device(T)
        terms = int((T.lengths().astype(np.int64) ** 2).sum())
        plan = crp.Plan(T.n_minor, T.n_minor, 64, ci.SEED_A, ci.SEED_B, flags=crp.CRP_PLAN_DIRECT,
                        stream=stream)

        def step():
            plan.reset()
            plan.accumulate(d, d)
            plan.sync()
            plan.topk(1000, upper=True)
        ms = _timed(step, args.steps, args.warmup, stream)
        acc_ms = plan.timing()[0]
        entries = plan.stats()["entries"]
        cpu = None if args.no_cpu else cpu_baseline(T, args.cpu_seconds)
        _line(terms / (ms / 1e3), ms, args, "i32",
              {"workload": "c1: 20000 transactions x 1000 items, Poisson(10) in [2,40], "
                           "Zipf(1.1); exact T^T T, P = 64, direct updates",
               "terms_per_step": terms, "accumulate_ms": acc_ms, "entries": entries},
              {"cpu_baseline": cpu,
               "roofline": _roofline(terms, d.nbytes(), entries, acc_ms, "k_accumulate (direct)")})
    elif args.workload == "c3":
        run_c3(args, np, torch, crp, ci, stream)
    elif args.workload == "c4":
        run_c4(args, np, torch, crp, ci, stream)
    else:
        run_c5(args, np, torch, crp, ci, stream)


def _roofline(terms, input_bytes, entries, kernel_ms, kernel):
    """The update roofline of the workload lines: one random read-modify-write
    of a 32-byte sector per term, the input read once, every entry written
    once, over the kernels' CUDA-event time, against the measured copy
    bandwidth."""
    hbm, peak_src = peaks()
    alg = terms * BYTES_PER_TERM_UPDATE + input_bytes + entries * SLOT_BYTES
    achieved = alg / (kernel_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "kernel": kernel, "kernel_ms": kernel_ms,
            "bytes_model": f"{BYTES_PER_TERM_UPDATE:g} B/term + input + {SLOT_BYTES:g} B/entry",
            "peak_source": f"{peak_src} hbm_gbs"}


def run_c3(args, np, torch, crp, ci, stream):
    """Real-valued C = A A (Markov-cluster expansion step).  Every variant of
    the fp32 accumulation is timed: the on-chip table (each CTA sums the exact
    products p + e of an entry as a compensated fp32 pair, TwoSum, and flushes
    the pair to the fp64 entry), direct updates and the routed variant (each
    product, exact in fp64, added to the fp64 entry with an atomic); the
    autotuner's choice is the line's value.  All stay within 1e-6 of the fp64
    oracle (tests)."""
    A, At = ci.c3()
    dA, dAt = crp.to_device(A), crp.to_device(At)
    terms = int((A.lengths().astype(np.int64) * At.lengths().astype(np.int64)).sum())
    kw, tps = crp.autotune(dA, dAt, A.n_minor, At.n_minor, ci.SEED_A, ci.SEED_B,
                           value_type=crp.CRP_F32_COMP, stream=stream)
    variants = {"autotuned": kw,
                "on_chip_twosum": dict(P=kw["P"], groups=1, flags=0),
                "direct_fp64_atomics": dict(P=kw["P"], flags=crp.CRP_PLAN_DIRECT),
                "routed_fp64_atomics": dict(P=kw["P"], flags=crp.CRP_PLAN_ROUTED)}
    out = {}
    for name, v in variants.items():
        plan = crp.Plan(A.n_minor, At.n_minor, seed_a=ci.SEED_A, seed_b=ci.SEED_B,
                        value_type=crp.CRP_F32_COMP, auto_grow=True, stream=stream, **v)

        def step():
            plan.reset()
            plan.accumulate(dA, dAt)
            plan.sync()
            plan.topk(1000)
        ms = _timed(step, args.steps, args.warmup, stream)
        st = plan.stats()
        out[name] = {"ms_per_step": ms, "accumulate_ms": plan.timing()[0],
                     "entries": st["entries"], "config": v}
        plan.close()
    best = out["autotuned"]
    cpu = None if args.no_cpu else cpu_baseline_real(A, At, args.cpu_seconds)
    _line(terms / (best["ms_per_step"] / 1e3), best["ms_per_step"], args, "f32/f64",
          {"workload": "c3: C = A A, A 100000 x 100000 column-stochastic, column nnz ~ "
                       "c^-2.1 on [5,2000], lognormal values; exact fp32 products, fp64 "
                       "entries",
           "terms_per_step": terms, "entries": best["entries"], "autotune": kw,
           "variants": out},
          {"cpu_baseline": cpu,
           "roofline": _roofline(terms, dA.nbytes() + dAt.nbytes(), best["entries"],
                                 best["accumulate_ms"], "k_accumulate (autotuned variant)")})


def cpu_baseline_real(A, At, budget_s: float):
    """The oracle, as it stands, on the first outer products of A A (doubled
    until one pass takes 2/3 of budget_s)."""
    from oracle import crp_oracle as O
    m = 1000
    while True:
        sa = O.Compressed(A.ptr[:m + 1], A.idx[:A.ptr[m]], A.val[:A.ptr[m]], A.n_minor)
        sb = O.Compressed(At.ptr[:m + 1], At.idx[:At.ptr[m]], At.val[:At.ptr[m]], At.n_minor)
        t0 = time.perf_counter()
        prod = O.exact_product(sa, sb, O.FULL)
        dt = time.perf_counter() - t0
        if dt >= budget_s * 2 / 3 or m * 2 > A.n_major:
            break
        m *= 2
    return {"value": prod.terms / dt, "unit": "terms/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m} outer products ({prod.terms} terms, {len(prod.i)} entries), "
                      f"{dt:.2f} s single-threaded numpy, fp64"}


def run_c4(args, np, torch, crp, ci, stream):
    """Heavy-entry mode: per-partition summaries with 2^20 counters over P = 256
    partitions (pairs i < j): plain, and with 2^16 reserved exact counters chosen
    by the product of marginals or by the trained network.  The top-1000 weight
    error of every variant is judged by the oracle's certified heaviest pairs
    of this input (tests/golden/c4_top16384.txt); for a scaled workload, which
    has no fixture, by the GPU exact product (which the tests pin bit-exact to
    the oracle) and labelled so."""
    w4 = ci.C4 if args.m is None else ci.C4.scaled(m=args.m)
    T = w4.generate()
    n = T.n_minor
    d = crp.to_device(T)
    m_pre = T.n_major // 100
    pre = crp.to_device(ci.Sparse(T.ptr[:m_pre + 1], T.idx[:T.ptr[m_pre]], None, n))
    L = T.lengths().astype(np.int64)
    terms = int((L * (L - 1) // 2).sum())
    rows, why = oracle_top_pairs("c4", T) if args.m is None else (None, "scaled workload")
    exact_ms = None
    if rows is None:
        ex = crp.Plan(n, n, 1024, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER,
                      flags=crp.CRP_PLAN_ROUTED | crp.CRP_PLAN_SORTED_ROWS,
                      hot_items=2048, warm_items=32, auto_grow=True, stream=stream)
        ex.accumulate(d, d)
        ex.sync()
        exact_ms = ex.timing()[0]
        gi, gj, gw, _ = ex.topk(8192, upper=True)
        ex.close()
        rows = list(zip(gi.tolist(), gj.tolist(), gw.tolist()))
        judged_by = f"GPU exact plan, top-8192 ({why})"
    else:
        judged_by = None
    ri = np.array([a for a, _, _ in rows[:1000]], np.int64)
    rj = np.array([b for _, b, _ in rows[:1000]], np.int64)
    rw = np.array([c for _, _, c in rows[:1000]], np.float64)
    top_sum = rw.sum()

    def judge(ti, tj):
        out = topk_weight_error(ti, tj, rows, 1000)
        if judged_by:
            out["judged_by"] = judged_by
        return out

    # network trained on a separate stream of the same recipe; labels are the
    # exact pair counts of that stream (GPU exact product)
    tr = ci.transactions(w4.seed + 17, 1_000_000, n, w4.lam, w4.lmin, w4.lmax, w4.zipf_s)
    dtr = crp.to_device(tr)
    ep = crp.Plan(n, n, 256, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER, flags=crp.CRP_PLAN_DIRECT,
                  auto_grow=True, stream=stream)
    ep.accumulate(dtr, dtr)
    ep.sync()
    ei, ej, ew, _ = ep.export()
    ep.close()
    keys = ei.astype(np.int64) * n + ej
    o = np.argsort(keys)
    keys, ew = keys[o], ew[o]
    R = 2048
    m_tp = tr.n_major // 100
    cpre = crp.to_device(ci.Sparse(tr.ptr[:m_tp + 1], tr.idx[:tr.ptr[m_tp]], None, n))
    cI, cJ, X = crp.candidate_pairs(cpre, n, R)
    ck = cI.cpu().numpy().astype(np.int64) * n + cJ.cpu().numpy()
    pos = np.minimum(np.searchsorted(keys, ck), len(keys) - 1)
    y = np.log1p(np.where(keys[pos] == ck, ew[pos], 0.0))
    Y = torch.tensor(y / max(y.max(), 1e-9), dtype=torch.float32, device="cuda")
    params = crp.mlp_init(7)
    trainer = crp.MLPTrainer(params, lr=3e-3)
    t0 = time.time()
    losses = [trainer.step(X, Y) for _ in range(300)]
    train_s = time.time() - t0
    results = {}
    qi = torch.from_numpy(ri.astype(np.int32)).cuda()
    qj = torch.from_numpy(rj.astype(np.int32)).cuda()
    for name, prm, reserve, sketch in (("plain", None, False, False),
                                       ("plain+sketch", None, False, True),
                                       ("product_of_marginals", None, True, False),
                                       ("predictor", params, True, False)):
        flags = crp.CRP_PLAN_SORTED_ROWS | (crp.CRP_PLAN_SKETCH if sketch else 0)
        plan = crp.Plan(n, n, 256, ci.SEED_A, ci.SEED_B, mode=crp.CRP_UPPER,
                        summary_counters=1 << 20, reserved_counters=(1 << 16) if reserve else 0,
                        flags=flags, stream=stream)
        t0 = time.time()
        if reserve:
            crp.predict_reserve(plan, pre, n, prm, R, 1 << 16)
        predict_s = time.time() - t0
        # warm-up passes, then the mean of timed passes (a reset keeps the
        # reserved keys)
        walls, kms = [], []
        for rep in range(args.warmup + args.steps):
            plan.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.accumulate(d, d)
            plan.sync()
            ti, tj, tw, tl = plan.topk(1000, upper=True)
            wall = time.perf_counter() - t0
            if rep >= args.warmup:
                walls.append(wall)
                kms.append(plan.timing()[0])
        wall = sum(walls) / len(walls)
        st = plan.stats()
        results[name] = {"terms_per_s": terms / wall, "seconds": wall,
                         "accumulate_kernel_ms": sum(kms) / len(kms),
                         "table_slots": st["table_slots"],
                         "top1000": judge(ti, tj),
                         "top1000_weight_err": judge(ti, tj)["topk_weight_err"],
                         "predict_reserve_s": predict_s, "passes": len(walls)}
        if sketch:
            # Count-Sketch estimates of the true top-1000 pairs: this
            # instance, and the median over 5 instances with independent seeds
            # (the other 4 run one at a time, untimed)
            ests = [crp.sketch_estimate([plan], qi, qj).cpu().numpy()]
            plan.close()
            for r in range(1, 5):
                extra = crp.Plan(n, n, 256, ci.SEED_A + 2 * r, ci.SEED_B + 2 * r + 1,
                                 mode=crp.CRP_UPPER, summary_counters=1 << 20, flags=flags,
                                 stream=stream)
                extra.accumulate(d, d)
                extra.sync()
                ests.append(crp.sketch_estimate([extra], qi, qj).cpu().numpy())
                extra.close()
            rel = [float(np.abs(e - rw).sum() / top_sum) for e in ests]
            med = np.median(np.array(ests), axis=0)
            results[name]["sketch_top1000_rel_err_one"] = rel[0]
            results[name]["sketch_top1000_rel_err_median5"] = float(np.abs(med - rw).sum() / top_sum)
        else:
            plan.close()
    regime = c4_paper_regime(args, np, torch, crp, ci, stream, d, n, terms, ri, rj, rw, top_sum,
                             judge, T) if args.paper_regime else None
    best = results["predictor"]
    cpu = None if args.no_cpu else cpu_baseline(T, args.cpu_seconds, mode=1)
    # roofline of the summary kernels: one random read-modify-write of a
    # 32-byte sector per term, the input read once, every summary slot
    # written once (compaction)
    hbm, peak_src = peaks()
    alg = terms * BYTES_PER_TERM_UPDATE + d.nbytes() + best["table_slots"] * SLOT_BYTES
    achieved = alg / (best["accumulate_kernel_ms"] / 1e3) / 1e9
    _line(best["terms_per_s"], best["seconds"] * 1e3, args, "u32 counters",
          {"workload": f"c4: {w4.m} transactions x {w4.n} items, Poisson(15), Zipf(1.2); "
                       "pairs i < j; 2^20 counters per partition, P = 256, 2^16 reserved "
                       "counters",
           "terms_per_step": terms, "exact_reference_ms": exact_ms,
           "top1000_judged_by": judged_by or "oracle certified top-16384 (tests/golden)",
           "training": {"samples": int(len(y)), "steps": 300, "first_loss": losses[0],
                        "last_loss": losses[-1], "seconds": train_s},
           "variants": results, "paper_regime": regime},
          {"cpu_baseline": cpu,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": None,
                        "kernel": "k_accumulate<summary>+k_summary_compact",
                        "kernel_ms": best["accumulate_kernel_ms"],
                        "bytes_model": f"{BYTES_PER_TERM_UPDATE:g} B/term + input + "
                                       f"{SLOT_BYTES:g} B/summary slot",
                        "peak_source": f"{peak_src} hbm_gbs"}})


def _bound_metrics(np, tw, tl):
    """From a list ranked by upper bound: the mean lower/upper ratio of its
    first 100 pairs (Figure 1(b)) and how many pairs come before the 100th
    whose lower bound is under 90 % of its upper bound (Section 6, larger
    Space-Saving structures; capped at the list's length)."""
    ratio = float(np.mean(tl[:100] / tw[:100]))
    bad = np.flatnonzero(tl < 0.9 * tw)
    until = int(bad[99]) if len(bad) >= 100 else int(len(tw))
    return ratio, until


def regime_cpu_baseline(T, budget_s: float):
    """The oracle, as it stands, on a prefix of the workload: one Space-Saving
    summary of 2 counters per bucket over 2^20 buckets, the canonical stream
    order (pairs i < j), and beside it the exact product and its per-bucket
    Count-Sketch; the prefix doubles until one pass takes 2/3 of budget_s."""
    from oracle import crp_oracle as O
    import crp_inputs as ci
    m = 1000
    while True:
        sub = O.Compressed(T.ptr[:m + 1], T.idx[:T.ptr[m]], None, T.n_minor)
        t0 = time.perf_counter()
        O.bucket_summaries(sub, sub, 1 << 20, 2, ci.SEED_A, ci.SEED_B, O.UPPER)
        t1 = time.perf_counter()
        prod = O.exact_product(sub, sub, O.UPPER)
        O.count_sketch(prod, 1 << 20, ci.SEED_A, ci.SEED_B)
        t2 = time.perf_counter()
        if t2 - t0 >= budget_s * 2 / 3 or m * 2 > T.n_major:
            break
        m *= 2
    return {"value": prod.terms / (t1 - t0), "unit": "terms/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m} transactions ({prod.terms} pairs i < j): bucket summaries "
                      f"{t1 - t0:.2f} s; exact product + Count-Sketch {t2 - t1:.2f} s "
                      f"({prod.terms / (t2 - t1):.3g} terms/s), single-threaded numpy"}


def c4_paper_regime(args, np, torch, crp, ci, stream, d, n, terms, ri, rj, rw, top_sum,
                    judge, T):
    """The paper's own summary regime (Section 6): many buckets (partitions)
    of two Space-Saving counters each, locked buckets updated in arrival
    order, with the Count-Sketch beside them.  Timed passes of P = 2^20,
    ell = 2 (on-chip combining before the buckets; and direct updates with
    the dense tiers counting pairs of frequent items); bucket count swept at ell = 2;
    ell swept at a fixed total of 2^21 counters; 11 instances with majority
    reporting (pairs in the top 3000 of at least 6) and median estimates."""
    F = crp.CRP_PLAN_LOCKED_SUMMARY | crp.CRP_PLAN_SORTED_ROWS
    out = {}

    def one(P, ell, seeds=(ci.SEED_A, ci.SEED_B), hot=0, warm=0, sketch=False, timed=0):
        fl = F | (crp.CRP_PLAN_SKETCH if sketch else 0) | (crp.CRP_PLAN_DIRECT if hot else 0)
        plan = crp.Plan(n, n, P, seeds[0], seeds[1], mode=crp.CRP_UPPER, summary_counters=ell,
                        flags=fl, hot_items=hot, warm_items=warm, stream=stream)
        walls = []
        for rep in range(1 + timed):
            plan.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.accumulate(d, d)
            plan.sync()
            walls.append(time.perf_counter() - t0)
        return plan, (sum(walls[1:]) / len(walls[1:]) if timed else walls[0])

    for name, hot, warm in (("P2^20_l2", 0, 0), ("P2^20_l2_tiers", 2048, 32)):
        plan, wall = one(1 << 20, 2, hot=hot, warm=warm, timed=max(args.steps, 1))
        tw_ = plan.topk(8192, upper=True)
        ratio, until = _bound_metrics(np, tw_[2], tw_[3])
        ti, tj, tw, _ = plan.topk(1000, upper=True)
        out[name] = {"terms_per_s": terms / wall, "seconds": wall,
                     "accumulate_kernel_ms": plan.timing()[0],
                     "top1000_weight_err": judge(ti, tj)["topk_weight_err"],
                     "top100_lower_over_upper": ratio, "pairs_until_100th_bad": until}
        plan.close()
    sweep = {}
    for lg in (14, 16, 18, 20):
        plan, wall = one(1 << lg, 2)
        tw_ = plan.topk(8192, upper=True)
        ratio, until = _bound_metrics(np, tw_[2], tw_[3])
        sweep[f"P2^{lg}"] = {"top100_lower_over_upper": ratio, "pairs_until_100th_bad": until,
                             "seconds": wall}
        plan.close()
    out["buckets_sweep_l2"] = sweep
    sweep = {}
    for ell in (2, 4, 8, 16):
        plan, wall = one((1 << 21) // ell, ell)
        tw_ = plan.topk(8192, upper=True)
        ratio, until = _bound_metrics(np, tw_[2], tw_[3])
        sweep[f"l{ell}"] = {"P": (1 << 21) // ell, "top100_lower_over_upper": ratio,
                            "pairs_until_100th_bad": until, "seconds": wall}
        plan.close()
    out["ell_sweep_2^21_counters"] = sweep
    # 11 instances, majority reporting, median of the Space-Saving upper bounds
    # and of the Count-Sketch estimates over the instances that report a pair
    t, K = 11, 3000
    reports = {}
    plans = []
    for r in range(t):
        plan, _ = one(1 << 20, 2, seeds=(ci.SEED_A + 2 * r, ci.SEED_B + 2 * r + 1), sketch=True)
        ti, tj, tw, _ = plan.topk(K, upper=True)
        for a, b, w in zip(ti.tolist(), tj.tolist(), tw.tolist()):
            reports.setdefault(a * n + b, []).append(w)
        plans.append(plan)
    qi = torch.from_numpy(ri.astype(np.int32)).cuda()
    qj = torch.from_numpy(rj.astype(np.int32)).cuda()
    cs_med = crp.sketch_estimate(plans, qi, qj).cpu().numpy()
    for pl in plans:
        pl.close()
    got_ss = np.zeros(len(rw))
    got_cs = np.zeros(len(rw))
    for q, k in enumerate((ri.astype(np.int64) * n + rj).tolist()):
        if len(reports.get(k, [])) >= (t + 1) // 2:
            got_ss[q] = np.median(reports[k])
            got_cs[q] = cs_med[q]
    if not args.no_cpu:
        out["cpu_baseline"] = regime_cpu_baseline(T, args.cpu_seconds)
    out["majority_11"] = {
        "top_k_per_instance": K,
        "exact_top1000_reported": float(np.mean(got_ss > 0)),
        "median_ss_rel_err": float(np.abs(got_ss - rw).sum() / top_sum),
        "median_cs_rel_err": float(np.abs(got_cs - rw).sum() / top_sum),
        "reported_pairs": int(sum(1 for v in reports.values() if len(v) >= (t + 1) // 2))}
    return out


def run_c5(args, np, torch, crp, ci, stream):
    """Batched: many independent co-occurrence problems in one persistent,
    graph-captured launch, against one launch per problem."""
    ws = ci.c5_params(args.c5_problems, m_range=(100, args.c5_mmax))
    t0 = time.time()
    Ts = [w.generate() for w in ws]
    gen_s = time.time() - t0
    dev = [crp.to_device(T) for T in Ts]
    terms = sum(int((T.lengths().astype(np.int64) ** 2).sum()) for T in Ts)
    t0 = time.time()
    kw, tune_tps = crp.autotune_batch([(x, x) for x in dev], ci.SEED_A, ci.SEED_B,
                                      sample_probs=256, stream=stream)
    tune_s = time.time() - t0
    batch = crp.Batch([(x, x) for x in dev], kw["P"], ci.SEED_A, ci.SEED_B,
                      tile_vectors=kw["tile_vectors"], hot_items=kw.get("hot_items", 0),
                      stream=stream)
    info = batch.info()

    def step():
        batch.run()
        batch.sync()
    ms = _timed(step, args.steps, args.warmup, stream)
    ev_ms, ev_terms = batch.sync()
    entries = [batch.count(q) for q in range(len(Ts))]
    batch.close()
    del batch
    # the same launch with the fixed choice used before tuning (P 256, 32 outer
    # products per work item), for comparison
    fixed = crp.Batch([(x, x) for x in dev], 256, ci.SEED_A, ci.SEED_B, tile_vectors=32,
                      stream=stream)

    def step_fixed():
        fixed.run()
        fixed.sync()
    ms_fixed = _timed(step_fixed, args.steps, args.warmup, stream)
    fixed.close()
    del fixed
    # baseline: one plan per problem, launched back to back (plans built first,
    # each sized from its problem's entry count)
    plans = [crp.Plan(T.n_minor, T.n_minor, 256, ci.SEED_A, ci.SEED_B, flags=crp.CRP_PLAN_DIRECT,
                      capacity_hint=int(e / 0.6) + 256 * 64, stream=stream)
             for T, e in zip(Ts, entries)]
    for p, x in zip(plans, dev):
        p.accumulate(x, x)
    for p in plans:
        p.sync()

    def per_problem():
        for p, x in zip(plans, dev):
            p.reset()
            p.accumulate(x, x)
        for p in plans:
            p.sync()
    ms_pp = _timed(per_problem, max(1, args.steps // 2), 1, stream)
    for p in plans:
        p.close()
    cpu = None if args.no_cpu else cpu_baseline_batch(Ts, args.cpu_seconds)
    input_bytes = sum(int(x.nbytes()) for x in dev)
    _line(terms / (ms / 1e3), ms, args, "i32",
          {"workload": f"c5: {len(ws)} problems, transactions log-U[100,{args.c5_mmax}], items "
                       "log-U[1e3,1e5], Zipf s ~ U[0.8,1.3], Poisson(12); exact T^T T each, "
                       "one persistent graph-captured launch",
           "terms_per_step": terms, "table_slots": info["table_slots"],
           "entries": int(sum(entries)), "generation_s": gen_s,
           "autotune": {"choice": kw, "sample_terms_per_s": tune_tps, "sample_problems": 256,
                        "seconds": round(tune_s, 1)},
           "fixed_P256_tile32": {"terms_per_s": terms / (ms_fixed / 1e3), "ms": ms_fixed}},
          {"one_launch_per_problem": {"terms_per_s": terms / (ms_pp / 1e3), "ms": ms_pp},
           "speedup_vs_per_problem": ms_pp / ms, "cpu_baseline": cpu,
           "roofline": _roofline(terms, input_bytes, int(sum(entries)), ev_ms,
                                 "k_batch (table reset + persistent launch)")})


def cpu_baseline_batch(Ts, budget_s: float):
    """The oracle, as it stands, on the batch's problems in order until about
    budget_s seconds of work (single thread)."""
    from oracle import crp_oracle as O
    t0 = time.perf_counter()
    terms = done = 0
    for T in Ts:
        Tc = O.Compressed.of(T)
        terms += O.exact_product(Tc, Tc, O.FULL).terms
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": terms / dt, "unit": "terms/s", "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {len(Ts)} problems ({terms} terms), {dt:.2f} s "
                      "single-threaded numpy"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "c2":
        run_other(args)
        return
    import numpy as np
    import torch
    import crp_inputs as ci
    import paper_1210_0461_gb300 as pkg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    pkg.build()
    from paper_1210_0461_gb300 import crp
    from paper_1210_0461_gb300.sharding import job_rate

    w = workload(args)
    t0 = time.time()
    T = w.generate()
    gen_s = time.time() - t0
    L = T.lengths()
    terms_step = int((L.astype(np.int64) ** 2).sum())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dT = crp.to_device(T, f"cuda:{local}")
    torch.cuda.synchronize()
    flags = crp.CRP_PLAN_NO_WARP_MATCH if args.no_match else 0
    flags |= {"direct": crp.CRP_PLAN_DIRECT, "smem": 0, "routed": crp.CRP_PLAN_ROUTED}[args.mode]

    tuned = None
    if args.autotune:
        t0 = time.time()
        if rank == 0:
            # results are cached per kernel version in the temp directory, so a
            # second run of the same command (under a profiler, say) times the
            # same configuration
            import tempfile
            cache = os.path.join(tempfile.gettempdir(), f"crp_tune_{kernel_source_hash()}.txt")
            kw, tps = crp.autotune(dT, dT, T.n_minor, T.n_minor, ci.SEED_A, ci.SEED_B,
                                   sample_vectors=min(args.autotune, T.n_major),
                                   cache_path=cache, stream=stream)
        if world > 1:   # every rank runs rank 0's choice
            box = [(kw, tps) if rank == 0 else None]
            torch.distributed.broadcast_object_list(box, src=0)
            kw, tps = box[0]
        tuned = {"choice": kw, "sample_terms_per_s": tps, "sample_vectors": args.autotune,
                 "seconds": round(time.time() - t0, 1)}
        args.P, args.groups, args.tile, args.smem_slots = (kw["P"], kw["groups"],
                                                           kw["tile_vectors"], kw["smem_slots"])
        args.hot = kw["hot_items"]
        args.warm = kw.get("warm_items", 0)
        flags = kw["flags"] | (crp.CRP_PLAN_NO_WARP_MATCH if args.no_match else 0)
        args.mode = ("routed" if flags & crp.CRP_PLAN_ROUTED else
                     "direct" if flags & crp.CRP_PLAN_DIRECT else "smem")
    # With N ranks, rank r owns partitions [r P / N, (r + 1) P / N) and reads the
    # whole input (Section 4: K instances on disjoint intervals, no exchange while
    # accumulating); the per-rank top-k lists are gathered and merged at the end.
    if args.sketch:
        flags |= crp.CRP_PLAN_SKETCH
    q, r = (0, 0)
    if world > 1:
        from paper_1210_0461_gb300.sharding import gather_topk, partition_interval
        q, r = partition_interval(rank, world, args.P)
    plan = crp.Plan(T.n_minor, T.n_minor, args.P, ci.SEED_A, ci.SEED_B, groups=args.groups,
                    tile_vectors=args.tile, smem_slots=args.smem_slots, flags=flags,
                    hot_items=args.hot, warm_items=args.warm, target_load_pct=args.load,
                    auto_grow=True, part_begin=q, part_end=r, stream=stream)

    def step():
        plan.reset()
        plan.accumulate(dT, dT)
        plan.sync()
        top = plan.topk(args.topk, upper=True)
        if world > 1:
            top = gather_topk(top[:3], args.topk)
        return top

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    launches0 = plan.timing()[1]

    # ---- timed region: K steps, inputs resident in HBM ----
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    acc_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        acc_ms.append(plan.timing()[0])
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = plan.timing()[1] - launches0
    st = plan.stats(per_partition=False)
    # the ranks split one product (each enumerates its own partition
    # interval): the job's terms are terms_step, over the slowest rank's time
    value, ms_step = job_rate(terms_step, ms_total / args.steps)

    # ---- roofline of the dominant kernel (k_accumulate) ----
    hbm, peak_src = peaks()
    acc = statistics.mean(acc_ms)
    entries = st["entries"]
    alg_bytes = (terms_step * BYTES_PER_TERM_UPDATE + dT.nbytes() + entries * SLOT_BYTES)
    achieved = alg_bytes / (acc / 1e3) / 1e9
    # DRAM bytes are captured with ncu only on cases within the profiling rules
    # (a few GB on the device); per term they grow with the table-to-L2 ratio, so
    # they are not scaled to this size (profiles/k_route_k_apply_c2_m500k.md)
    traffic = None
    # The atomic roofline: the accumulate's terms per second against the rate
    # of random 32-bit atomic adds (no return) into an L2-resident 16 MB region,
    # measured here with the library's probe kernel. Every term outside the
    # shared-memory core costs at least one L2 atomic or store, so this rate
    # bounds the accumulate from above as the copy bandwidth does.
    l2_atomics = crp.probe_update_rate(16 << 20, 1 << 28, 0)
    atomic_roofline = {"terms_per_s": terms_step / (acc / 1e3), "peak_atomics_per_s": l2_atomics,
                       "frac": terms_step / (acc / 1e3) / l2_atomics,
                       "peak_source": "crp_probe_update_rate: 2^28 random 32-bit atomic adds "
                                      "into a 16 MB region, timed in this run"}

    # ---- end to end through the C ABI from pinned host buffers ----
    # Every step copies its input from pinned host memory and reads its top-k
    # back to the host. The input goes into one of two device buffers: the copy
    # for step s + 1 runs on its own stream while step s computes from the
    # other buffer (it waits for the step that last read its buffer), so the
    # timed region holds every step's copy, overlapped with the step before.
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(T.ptr).pin_memory()
        hi = torch.from_numpy(T.idx).pin_memory()
        dev = f"cuda:{local}"
        bufs = [(torch.empty_like(hp, device=dev), torch.empty_like(hi, device=dev))
                for _ in range(2)]
        dds = [crp.DeviceSparse(bp, bi, None, T.n_minor) for bp, bi in bufs]
        copy_stream = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        released = [torch.cuda.Event(), torch.cuda.Event()]
        for e in released:
            e.record(stream)

        def issue_copy(slot):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(released[slot])
                bufs[slot][0].copy_(hp, non_blocking=True)
                bufs[slot][1].copy_(hi, non_blocking=True)
                copied[slot].record(copy_stream)

        def e2e_run(n):
            issue_copy(0)
            top = None
            for s_ in range(n):
                slot = s_ & 1
                if s_ + 1 < n:
                    issue_copy(slot ^ 1)
                plan.reset()
                stream.wait_event(copied[slot])
                plan.accumulate(dds[slot], dds[slot])
                released[slot].record(stream)
                plan.sync()
                top = plan.topk(args.topk, upper=True)   # host outputs: D2H inside
                if world > 1:
                    top = gather_topk(top[:3], args.topk)
            return top

        e2e_run(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        torch.cuda.synchronize()
        e_rate, e_ms = job_rate(terms_step, (time.perf_counter() - t0) * 1e3 / args.steps)
        e2e = {"value": e_rate, "unit": "terms/s",
               "h2d_bytes_per_step": int(hp.numel() * 8 + hi.numel() * 4),
               "d2h_bytes_per_step": int(args.topk * (4 + 4 + 8 + 8)), "ms_per_step": e_ms,
               "copies": "each step's input copied from pinned host memory into one of two "
                         "device buffers while the step before computes; top-k read back "
                         "to host memory every step"}

    ti, tj, tw, _ = plan.topk(args.topk, upper=True)
    # the top-k judged by the oracle's certified heaviest pairs of this input
    judged = {"topk_weight_err": None}
    if rank == 0 and args.m is None:
        rows, why = oracle_top_pairs("c2", T)
        judged = (topk_weight_error(ti, tj, rows, args.topk) if rows
                  else {"topk_weight_err": None, "why": why})
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(T, args.cpu_seconds)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.m} transactions x {w.n} items, Poisson"
                                   f"({w.lam:g}) in [{w.lmin},{w.lmax}], Zipf({w.zipf_s:g}); "
                                   "exact int32 T^T T (all entries), top-1000 pairs",
                       "P": args.P, "groups": args.groups, "tile_vectors": args.tile,
                       "smem_slots": args.smem_slots, "warp_match": not args.no_match,
                       "mode": args.mode, "hot_items": args.hot, "warm_items": args.warm,
                       "target_load_pct": args.load, "count_sketch": bool(args.sketch),
                       "topk_from_hot_block": plan.topk_certified_calls(),
                       "autotune": tuned,
                       "terms_per_step": terms_step, "entries": entries,
                       "nnz": int(T.nnz), "l2": "inputs (0.8 GB) and tables "
                       f"({st['table_slots'] * 16 / 1e9:.1f} GB) exceed L2; no flush",
                       "step": "reset + accumulate + sync + topk",
                       "parallelism": (f"partition intervals: {world} ranks x {args.P // world} "
                                       "partitions, input replicated, top-k gathered")
                       if world > 1 else "one GPU",
                       "topk_weight_err": judged.get("topk_weight_err"),
                       "topk_judged": judged,
                       "gen_seconds": round(gen_s, 2)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": {"direct": "k_accumulate", "smem": "k_accumulate",
                                    "routed": "k_route+k_apply_bulk"}[args.mode]
                                   + ("+k_hot_flush" if args.hot else "")
                                   + ("+k_warm_flush" if args.warm else ""),
                         "kernel_ms": acc,
                         "route_ms": st.get("last_route_ms"),
                         "bytes_model": f"{BYTES_PER_TERM_UPDATE:g} B/term + input + "
                                        f"{SLOT_BYTES:g} B/entry",
                         "peak_source": f"{peak_src} hbm_gbs"},
            "atomic_roofline": atomic_roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "top_pair": [int(ti[0]), int(tj[0]), float(tw[0])] if len(ti) else None,
            "combine_ratio": st["terms"] / max(st["flushed_updates"], 1),
        }
        print(json.dumps(out), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
