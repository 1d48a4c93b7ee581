"""ctypes binding of libcrp (include/crp.h): argument marshalling only.

Every step of the product runs in the CUDA kernels of libcrp.so; this module
only builds the C structs, passes device pointers taken from torch tensors and
the current torch stream, and turns status codes into exceptions.  There is no
CPU path: if the library is missing the import of :func:`lib` fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcrp.so")

CRP_OK, CRP_EINVAL, CRP_ENOMEM, CRP_ETABLE_FULL, CRP_ETIMEOUT, CRP_ECUDA, CRP_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "CRP_OK", 1: "CRP_EINVAL", 2: "CRP_ENOMEM", 3: "CRP_ETABLE_FULL",
                4: "CRP_ETIMEOUT", 5: "CRP_ECUDA", 6: "CRP_EUNSUPPORTED"}
CRP_I32, CRP_F32_COMP = 0, 1
CRP_FULL, CRP_UPPER = 0, 1
CRP_TOPK_UPPER = 1
CRP_PLAN_NO_WARP_MATCH, CRP_PLAN_DEBUG_CHECKS, CRP_PLAN_DIRECT, CRP_PLAN_ROUTED = 1, 2, 4, 8
CRP_PLAN_SORTED_ROWS = 16
CRP_PLAN_SKETCH = 32
CRP_PLAN_LOCKED_SUMMARY = 64


class CrpError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class crp_sparse(ctypes.Structure):
    _fields_ = [("n_major", ctypes.c_int64), ("n_minor", ctypes.c_int32),
                ("_pad", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("ptr", ctypes.c_void_p), ("idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class crp_plan_desc(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
                ("P", ctypes.c_uint32), ("_pad0", ctypes.c_uint32),
                ("seed_a", ctypes.c_uint64), ("seed_b", ctypes.c_uint64),
                ("value_type", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("summary_counters", ctypes.c_uint32), ("reserved_counters", ctypes.c_uint32),
                ("table_capacity_hint", ctypes.c_uint64), ("auto_grow", ctypes.c_int32),
                ("groups", ctypes.c_uint32), ("tile_vectors", ctypes.c_uint32),
                ("smem_slots", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("hot_items", ctypes.c_uint32), ("target_load_pct", ctypes.c_uint32),
                ("part_begin", ctypes.c_uint32), ("part_end", ctypes.c_uint32),
                ("warm_items", ctypes.c_uint32), ("route_pool_chunks", ctypes.c_uint32),
                ("lock_wait_us", ctypes.c_uint32)]


class crp_stats_t(ctypes.Structure):
    _fields_ = [("terms", ctypes.c_uint64), ("flushed_updates", ctypes.c_uint64),
                ("entries", ctypes.c_uint64), ("table_slots", ctypes.c_uint64),
                ("spilled", ctypes.c_uint64), ("full_partitions", ctypes.c_uint32),
                ("P", ctypes.c_uint32), ("max_over_mean_terms", ctypes.c_double),
                ("last_accumulate_ms", ctypes.c_double), ("launches", ctypes.c_uint64),
                ("last_route_ms", ctypes.c_double), ("estimated_entries", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "crp_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(crp_plan_desc), _P]),
    "crp_plan_destroy": (None, [_P]),
    "crp_reset": (ctypes.c_int, [_P]),
    "crp_outer_accumulate": (ctypes.c_int, [_P, ctypes.POINTER(crp_sparse),
                                            ctypes.POINTER(crp_sparse)]),
    "crp_sync": (ctypes.c_int, [_P]),
    "crp_topk": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, _P, _P, _P, _P,
                                ctypes.POINTER(ctypes.c_int32)]),
    "crp_partition_of": (ctypes.c_uint32, [_P, ctypes.c_int32, ctypes.c_int32]),
    "crp_topk_certified_calls": (ctypes.c_uint64, [_P]),
    "crp_reserve": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "crp_export_partitions": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32, _P, _P, _P, _P,
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "crp_stats": (ctypes.c_int, [_P, ctypes.POINTER(crp_stats_t), _P]),
    "crp_timing": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "crp_probe_update_rate": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_double)]),
    "crp_outer_product_noalloc": (ctypes.c_int, [ctypes.POINTER(crp_plan_desc),
                                                 ctypes.POINTER(crp_sparse),
                                                 ctypes.POINTER(crp_sparse), _P, _P, _P,
                                                 ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                                 _P]),
    "crp_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(crp_plan_desc),
                                        ctypes.c_int32, _P, _P, ctypes.c_uint64, _P]),
    "crp_batch_run": (ctypes.c_int, [_P]),
    "crp_batch_sync": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "crp_batch_set_ready": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "crp_batch_export": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "crp_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "crp_batch_destroy": (None, [_P]),
    "crp_mlp_param_count": (ctypes.c_int32, []),
    "crp_mlp_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
    "crp_mlp_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P]),
    "crp_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_float, ctypes.c_int32, _P]),
    "crp_candidate_pairs": (ctypes.c_int, [ctypes.POINTER(crp_sparse), ctypes.c_int32,
                                           ctypes.c_int32, _P, _P, _P, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64), _P]),
    "crp_predict_reserve": (ctypes.c_int, [_P, ctypes.POINTER(crp_sparse), ctypes.c_int32, _P,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
    "crp_autotune": (ctypes.c_int, [ctypes.POINTER(crp_plan_desc), ctypes.POINTER(crp_sparse),
                                    ctypes.POINTER(crp_sparse), ctypes.c_int64, ctypes.c_char_p,
                                    ctypes.POINTER(crp_plan_desc),
                                    ctypes.POINTER(ctypes.c_double), _P]),
    "crp_autotune_batch": (ctypes.c_int, [ctypes.POINTER(crp_plan_desc), ctypes.c_int32, _P,
                                          _P, ctypes.c_int32, ctypes.c_char_p,
                                          ctypes.POINTER(crp_plan_desc),
                                          ctypes.POINTER(ctypes.c_double), _P]),
    "crp_sketch_read": (ctypes.c_int, [_P, _P]),
    "crp_sketch_estimate": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P]),
    "crp_debug_hold_lock": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "crp_version": (ctypes.c_char_p, []),
    "crp_last_error": (ctypes.c_char_p, []),
}


def exported_symbols() -> list[str]:
    return list(_SIGS)


def lib() -> ctypes.CDLL:
    """Load libcrp.so.  Raises when it has not been built (there is no
    fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libcrp.so is not built ({LIB_PATH}); run "
                                  "paper_1210_0461_gb300._build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != CRP_OK:
        raise CrpError(st, where, lib().crp_last_error().decode())


# ---------------------------------------------------------------------------
# Device-side inputs
# ---------------------------------------------------------------------------

@dataclass
class DeviceSparse:
    """K compressed vectors held in torch tensors on a CUDA device."""
    ptr: "object"     # torch.int64 [K+1]
    idx: "object"     # torch.int32 [nnz]
    val: "object"     # torch.float32 [nnz] or None
    n_minor: int

    @property
    def n_major(self) -> int:
        return int(self.ptr.shape[0]) - 1

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])

    def c_struct(self) -> crp_sparse:
        s = crp_sparse()
        s.n_major = self.n_major
        s.n_minor = self.n_minor
        s.nnz = self.nnz
        s.ptr = self.ptr.data_ptr()
        s.idx = self.idx.data_ptr() if self.nnz else 0
        s.val = self.val.data_ptr() if self.val is not None and self.nnz else None
        return s

    def nbytes(self) -> int:
        b = self.ptr.numel() * 8 + self.idx.numel() * 4
        return b + (self.val.numel() * 4 if self.val is not None else 0)


def to_device(sp, device="cuda", pin: bool = False) -> DeviceSparse:
    """Copy a host compressed matrix (any object with ptr, idx, val, n_minor
    numpy arrays) to the device."""
    import torch
    ptr = torch.from_numpy(np.ascontiguousarray(sp.ptr, dtype=np.int64))
    idx = torch.from_numpy(np.ascontiguousarray(sp.idx, dtype=np.int32))
    val = None if sp.val is None else torch.from_numpy(np.ascontiguousarray(sp.val, np.float32))
    if pin:
        ptr, idx = ptr.pin_memory(), idx.pin_memory()
        val = val.pin_memory() if val is not None else None
    return DeviceSparse(ptr.to(device, non_blocking=pin), idx.to(device, non_blocking=pin),
                        None if val is None else val.to(device, non_blocking=pin), int(sp.n_minor))


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ---------------------------------------------------------------------------
# Plan
# ---------------------------------------------------------------------------

class Plan:
    """An exact column-row product plan: P hash partitions, each with its own
    open-addressing table in device memory (see include/crp.h)."""

    def __init__(self, n_rows: int, n_cols: int, P: int, seed_a: int, seed_b: int,
                 value_type: int = CRP_I32, mode: int = CRP_FULL, groups: int = 0,
                 tile_vectors: int = 0, smem_slots: int = 0, capacity_hint: int = 0,
                 auto_grow: bool = False, flags: int = 0, stream=None,
                 summary_counters: int = 0, reserved_counters: int = 0, hot_items: int = 0,
                 target_load_pct: int = 0, part_begin: int = 0, part_end: int = 0,
                 warm_items: int = 0, route_pool_chunks: int = 0, lock_wait_us: int = 0):
        self._lib = lib()
        d = crp_plan_desc()
        d.n_rows, d.n_cols, d.P = n_rows, n_cols, P
        d.seed_a, d.seed_b = seed_a & (2**64 - 1), seed_b & (2**64 - 1)
        d.value_type, d.mode = value_type, mode
        d.table_capacity_hint = capacity_hint
        d.summary_counters, d.reserved_counters = summary_counters, reserved_counters
        d.hot_items = hot_items
        d.target_load_pct = target_load_pct
        d.part_begin, d.part_end = part_begin, part_end
        d.warm_items = warm_items
        d.route_pool_chunks, d.lock_wait_us = route_pool_chunks, lock_wait_us
        d.auto_grow = 1 if auto_grow else 0
        d.groups, d.tile_vectors, d.smem_slots, d.flags = groups, tile_vectors, smem_slots, flags
        self.desc = d
        self.P = P
        self.value_type = value_type
        self._stream = stream
        h = _P()
        _check(self._lib.crp_plan_create(ctypes.byref(h), ctypes.byref(d), _stream_handle(stream)),
               "crp_plan_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.crp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        _check(self._lib.crp_reset(self._h), "crp_reset")

    def accumulate(self, A: DeviceSparse, B: DeviceSparse):
        a, b = A.c_struct(), B.c_struct()
        _check(self._lib.crp_outer_accumulate(self._h, ctypes.byref(a), ctypes.byref(b)),
               "crp_outer_accumulate")
        if self.P == 0 and A.n_major > 0:   # tuned by the first call: learn its P
            s = crp_stats_t()
            _check(self._lib.crp_stats(self._h, ctypes.byref(s), None), "crp_stats")
            self.P = int(s.P)

    def sync(self):
        _check(self._lib.crp_sync(self._h), "crp_sync")

    def reserve(self, keys):
        """Register (i << 32 | j) keys for exact counting (summary mode)."""
        k = np.ascontiguousarray(keys, dtype=np.uint64)
        _check(self._lib.crp_reserve(self._h, k.ctypes.data if len(k) else None, len(k)),
               "crp_reserve")

    def debug_hold_lock(self, p: int):
        """Test hook: hold partition p's bucket lock (crp_debug_hold_lock)."""
        _check(self._lib.crp_debug_hold_lock(self._h, p), "crp_debug_hold_lock")

    def partition_of(self, i: int, j: int) -> int:
        return int(self._lib.crp_partition_of(self._h, i, j))

    def topk(self, k: int, upper: bool = False, device_out=None):
        """(i, j, w, w_lower) of the k heaviest entries, numpy arrays (or torch
        tensors on ``device_out``)."""
        n = ctypes.c_int32(0)
        flags = CRP_TOPK_UPPER if upper else 0
        if device_out is not None:
            import torch
            i = torch.empty(k, dtype=torch.int32, device=device_out)
            j = torch.empty(k, dtype=torch.int32, device=device_out)
            w = torch.empty(k, dtype=torch.float64, device=device_out)
            wl = torch.empty(k, dtype=torch.float64, device=device_out)
            ptrs = [t.data_ptr() for t in (i, j, w, wl)]
        else:
            i = np.zeros(k, np.int32)
            j = np.zeros(k, np.int32)
            w = np.zeros(k, np.float64)
            wl = np.zeros(k, np.float64)
            ptrs = [t.ctypes.data for t in (i, j, w, wl)]
        _check(self._lib.crp_topk(self._h, k, flags, *ptrs, ctypes.byref(n)), "crp_topk")
        m = n.value
        return i[:m], j[:m], w[:m], wl[:m]

    def topk_certified_calls(self) -> int:
        """crp_topk calls answered from the hot block alone (see include/crp.h)."""
        return int(self._lib.crp_topk_certified_calls(self._h))

    def export(self, p_begin: int = 0, p_end: int | None = None):
        """All entries of partitions [p_begin, p_end): (i, j, w, w_lower, counts
        per partition) as numpy arrays."""
        p_end = self.P if p_end is None else p_end
        n = ctypes.c_int64(0)
        st = self._lib.crp_export_partitions(self._h, p_begin, p_end, None, None, None, None, 0,
                                             ctypes.byref(n))
        if st not in (CRP_OK, CRP_EINVAL) or (st == CRP_EINVAL and n.value == 0):
            _check(st, "crp_export_partitions")
        cap = n.value
        i = np.zeros(cap, np.int32)
        j = np.zeros(cap, np.int32)
        w = np.zeros(cap, np.float64)
        wl = np.zeros(cap, np.float64)
        if cap:
            _check(self._lib.crp_export_partitions(self._h, p_begin, p_end, i.ctypes.data,
                                                   j.ctypes.data, w.ctypes.data, wl.ctypes.data,
                                                   cap, ctypes.byref(n)), "crp_export_partitions")
        return i, j, w, wl

    def timing(self):
        """(device ms of the last enumeration kernel, kernels launched so far)."""
        ms = ctypes.c_double(0)
        n = ctypes.c_uint64(0)
        _check(self._lib.crp_timing(self._h, ctypes.byref(ms), ctypes.byref(n)), "crp_timing")
        return ms.value, n.value

    def sketch(self) -> np.ndarray:
        """The Count-Sketch's P estimators (CRP_PLAN_SKETCH): int64 for
        CRP_I32 plans, float64 for CRP_F32_COMP plans."""
        out = np.zeros(self.P, np.int64 if self.value_type == CRP_I32 else np.float64)
        _check(self._lib.crp_sketch_read(self._h, out.ctypes.data), "crp_sketch_read")
        return out

    def stats(self, per_partition: bool = False):
        s = crp_stats_t()
        terms = np.zeros(self.P, np.uint64) if per_partition else None
        _check(self._lib.crp_stats(self._h, ctypes.byref(s),
                                   terms.ctypes.data if terms is not None else None), "crp_stats")
        d = {f: getattr(s, f) for f, _ in crp_stats_t._fields_}
        if per_partition:
            d["partition_terms"] = terms
        return d


def sketch_estimate(plans, i, j):
    """Median over the plans' Count-Sketches of the estimates of entries
    (i[q], j[q]); i, j: int32 CUDA tensors.  Returns a float64 CUDA tensor."""
    import torch
    i = i.to(torch.int32).contiguous()
    j = j.to(torch.int32).contiguous()
    out = torch.empty(i.numel(), dtype=torch.float64, device=i.device)
    arr = (_P * len(plans))(*[p._h for p in plans])
    _check(lib().crp_sketch_estimate(arr, len(plans), i.data_ptr(), j.data_ptr(), i.numel(),
                                     out.data_ptr()), "crp_sketch_estimate")
    return out


def probe_update_rate(region_bytes: int, n_updates: int, mode: int) -> float:
    """Updates per second of the random-update probe (see include/crp.h)."""
    ms = ctypes.c_double(0)
    _check(lib().crp_probe_update_rate(region_bytes, n_updates, mode, ctypes.byref(ms)),
           "crp_probe_update_rate")
    return n_updates / (ms.value / 1e3)


class Batch:
    """Many independent co-occurrence products in one persistent, graph-captured
    launch (crp_batch_* in include/crp.h).  ``problems``: list of
    (A, B) DeviceSparse pairs."""

    def __init__(self, problems, P: int, seed_a: int, seed_b: int, mode: int = CRP_FULL,
                 tile_vectors: int = 0, wait_timeout_ns: int = 0, hot_items: int = 0,
                 stream=None):
        self._lib = lib()
        d = crp_plan_desc()
        d.n_rows = d.n_cols = 1
        d.P, d.seed_a, d.seed_b = P, seed_a & (2**64 - 1), seed_b & (2**64 - 1)
        d.value_type, d.mode, d.tile_vectors = CRP_I32, mode, tile_vectors
        d.hot_items = hot_items
        n = len(problems)
        self._keep = problems
        A = (crp_sparse * n)(*[a.c_struct() for a, _ in problems])
        B = (crp_sparse * n)(*[b.c_struct() for _, b in problems])
        h = _P()
        _check(self._lib.crp_batch_create(ctypes.byref(h), ctypes.byref(d), n,
                                          ctypes.cast(A, _P), ctypes.cast(B, _P), wait_timeout_ns,
                                          _stream_handle(stream)), "crp_batch_create")
        self._h = h
        self.n = n

    def run(self):
        _check(self._lib.crp_batch_run(self._h), "crp_batch_run")

    def sync(self):
        ms = ctypes.c_double(0)
        t = ctypes.c_uint64(0)
        _check(self._lib.crp_batch_sync(self._h, ctypes.byref(ms), ctypes.byref(t)),
               "crp_batch_sync")
        return ms.value, t.value

    def set_ready(self, q: int, ready: bool):
        _check(self._lib.crp_batch_set_ready(self._h, q, 1 if ready else 0), "crp_batch_set_ready")

    def export(self, q: int):
        n = ctypes.c_int64(0)
        st = self._lib.crp_batch_export(self._h, q, None, None, None, 0, ctypes.byref(n))
        if st not in (CRP_OK, CRP_EINVAL):
            _check(st, "crp_batch_export")
        cap = n.value
        i = np.zeros(cap, np.int32)
        j = np.zeros(cap, np.int32)
        w = np.zeros(cap, np.float64)
        if cap:
            _check(self._lib.crp_batch_export(self._h, q, i.ctypes.data, j.ctypes.data,
                                              w.ctypes.data, cap, ctypes.byref(n)),
                   "crp_batch_export")
        return i, j, w

    def count(self, q: int) -> int:
        """Number of entries of problem q."""
        n = ctypes.c_int64(0)
        st = self._lib.crp_batch_export(self._h, q, None, None, None, 0, ctypes.byref(n))
        if st not in (CRP_OK, CRP_EINVAL):
            _check(st, "crp_batch_export")
        return n.value

    def info(self):
        t, s, l = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(self._lib.crp_batch_info(self._h, ctypes.byref(t), ctypes.byref(s),
                                        ctypes.byref(l)), "crp_batch_info")
        return {"total_terms": t.value, "table_slots": s.value, "launches": l.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.crp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Heavy-pair predictor (tcgen05 MLP)
# ---------------------------------------------------------------------------

def mlp_param_count() -> int:
    return int(lib().crp_mlp_param_count())


def mlp_forward(params, x):
    """y for the rows of x (torch tensors on the device: params fp32 [4417],
    x fp32 [n, 2])."""
    import torch
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().crp_mlp_forward(params.data_ptr(), x.data_ptr(), y.data_ptr(), x.shape[0],
                                 _stream_handle(None)), "crp_mlp_forward")
    return y


def mlp_grad(params, x, t, n_total=None):
    """(loss, grad) of sum (y - t)^2 / n_total (device tensors)."""
    import torch
    g = torch.empty(mlp_param_count(), dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    n = x.shape[0]
    _check(lib().crp_mlp_grad(params.data_ptr(), x.data_ptr(), t.data_ptr(), n,
                              n if n_total is None else n_total, g.data_ptr(), loss.data_ptr(),
                              _stream_handle(None)), "crp_mlp_grad")
    return float(loss.item()), g


def mlp_init(seed: int, device="cuda"):
    """Initial parameters (He-style normal weights, small positive biases) as a
    device tensor in the layout of crp_mlp_forward."""
    import torch
    g = np.random.default_rng(seed)
    parts = [g.normal(0, 1.0, 128), np.full(64, 0.01), g.normal(0, np.sqrt(2 / 64), 4096),
             np.full(64, 0.01), g.normal(0, np.sqrt(1 / 64), 64), np.zeros(1)]
    return torch.tensor(np.concatenate(parts), dtype=torch.float32, device=device)


def mlp_adam(params, m, v, grad, lr: float, step: int):
    """One Adam step on device tensors (params, m, v updated in place)."""
    _check(lib().crp_mlp_adam(params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(),
                              lr, step, _stream_handle(None)), "crp_mlp_adam")


class MLPTrainer:
    """Adam on the fp32 master parameters with the tensor-core gradient kernel."""

    def __init__(self, params, lr=1e-2):
        import torch
        self.params = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.lr = lr
        self.step_n = 0

    def step(self, x, t):
        loss, g = mlp_grad(self.params, x, t)
        self.step_n += 1
        mlp_adam(self.params, self.m, self.v, g, self.lr, self.step_n)
        return loss


def candidate_pairs(prefix: DeviceSparse, n_items: int, R: int):
    """(i, j, x) device tensors of the candidate pairs of a stream prefix."""
    import torch
    nc = R * (R - 1) // 2
    dev = prefix.idx.device
    i = torch.empty(nc, dtype=torch.int32, device=dev)
    j = torch.empty(nc, dtype=torch.int32, device=dev)
    x = torch.empty((nc, 2), dtype=torch.float32, device=dev)
    n = ctypes.c_int64(0)
    s = prefix.c_struct()
    _check(lib().crp_candidate_pairs(ctypes.byref(s), n_items, R, i.data_ptr(), j.data_ptr(),
                                     x.data_ptr(), nc, ctypes.byref(n), _stream_handle(None)),
           "crp_candidate_pairs")
    return i, j, x


def predict_reserve(plan: "Plan", prefix: DeviceSparse, n_items: int, params, R: int,
                    n_reserve: int, full_mode: bool = False):
    s = prefix.c_struct()
    _check(lib().crp_predict_reserve(plan._h, ctypes.byref(s), n_items,
                                     params.data_ptr() if params is not None else None, R,
                                     n_reserve, 1 if full_mode else 0, _stream_handle(None)),
           "crp_predict_reserve")


def autotune(A: DeviceSparse, B: DeviceSparse, n_rows: int, n_cols: int, seed_a: int, seed_b: int,
             value_type: int = CRP_I32, mode: int = CRP_FULL, sample_vectors: int = 0,
             cache_path: str | None = None, stream=None):
    """Fastest launch configuration for this input (see crp_autotune):
    returns (dict of Plan keyword arguments, terms/s measured)."""
    d = crp_plan_desc()
    d.n_rows, d.n_cols, d.P = n_rows, n_cols, 1024
    d.seed_a, d.seed_b = seed_a & (2**64 - 1), seed_b & (2**64 - 1)
    d.value_type, d.mode = value_type, mode
    best = crp_plan_desc()
    tps = ctypes.c_double(0)
    a, b = A.c_struct(), B.c_struct()
    _check(lib().crp_autotune(ctypes.byref(d), ctypes.byref(a), ctypes.byref(b), sample_vectors,
                              cache_path.encode() if cache_path else None, ctypes.byref(best),
                              ctypes.byref(tps), _stream_handle(stream)), "crp_autotune")
    kw = dict(P=best.P, groups=best.groups, tile_vectors=best.tile_vectors,
              smem_slots=best.smem_slots, flags=best.flags, hot_items=best.hot_items,
              warm_items=best.warm_items)
    return kw, tps.value


def autotune_batch(problems, seed_a: int, seed_b: int, mode: int = CRP_FULL,
                   sample_probs: int = 256, cache_path: str | None = None, stream=None):
    """Fastest (P, tile_vectors, hot_items) of the batched launch for these problems
    (crp_autotune_batch): returns (dict of Batch keyword arguments, terms/s on
    the sample)."""
    d = crp_plan_desc()
    d.n_rows = d.n_cols = 1
    d.P, d.seed_a, d.seed_b = 256, seed_a & (2**64 - 1), seed_b & (2**64 - 1)
    d.value_type, d.mode = CRP_I32, mode
    n = len(problems)
    A = (crp_sparse * n)(*[a.c_struct() for a, _ in problems])
    B = (crp_sparse * n)(*[b.c_struct() for _, b in problems])
    best = crp_plan_desc()
    tps = ctypes.c_double(0)
    _check(lib().crp_autotune_batch(ctypes.byref(d), n, ctypes.cast(A, _P), ctypes.cast(B, _P),
                                    sample_probs, cache_path.encode() if cache_path else None,
                                    ctypes.byref(best), ctypes.byref(tps),
                                    _stream_handle(stream)), "crp_autotune_batch")
    return dict(P=best.P, tile_vectors=best.tile_vectors, hot_items=best.hot_items), tps.value
