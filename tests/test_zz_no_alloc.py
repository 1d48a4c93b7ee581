"""The allocation-free entry point, crp_outer_product_noalloc.

It exists for callers that cannot call cudaMalloc (code under an external
memory manager that owns the device, regions where an allocation would
synchronise or is forbidden).  Its partition tables live in a static device
array, so two calls in a row share that array: each call must clear it and
still agree with the plan-based entry points (crp_plan_create +
crp_outer_accumulate + crp_export_partitions) on the same input.  This file is
collected last so a failure here cannot hide failures elsewhere."""
import ctypes

import numpy as np
import pytest

import crp_inputs as ci

pytestmark = pytest.mark.gpu

RTOL_REAL = 1e-6


@pytest.fixture(scope="module")
def crp():
    import torch
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp as c
    torch.cuda.init()
    return c


def _noalloc(crp, A, B, n_rows, n_cols, P, value_type, mode, capacity):
    import torch
    d = crp.crp_plan_desc()
    d.n_rows, d.n_cols, d.P = n_rows, n_cols, P
    d.seed_a, d.seed_b = ci.SEED_A, ci.SEED_B
    d.value_type, d.mode = value_type, mode
    dA = crp.to_device(A)
    dB = dA if B is A else crp.to_device(B)
    a, b = dA.c_struct(), dB.c_struct()
    i = torch.empty(capacity, dtype=torch.int32, device="cuda")
    j = torch.empty(capacity, dtype=torch.int32, device="cuda")
    w = torch.empty(capacity, dtype=torch.float64, device="cuda")
    n = ctypes.c_int64(0)
    stream = torch.cuda.current_stream().cuda_stream
    st = crp.lib().crp_outer_product_noalloc(ctypes.byref(d), ctypes.byref(a), ctypes.byref(b),
                                             i.data_ptr(), j.data_ptr(), w.data_ptr(), capacity,
                                             ctypes.byref(n), stream)
    assert st == crp.CRP_OK, crp.lib().crp_last_error()
    m = n.value
    return i[:m].cpu().numpy(), j[:m].cpu().numpy(), w[:m].cpu().numpy()


def _with_plan(crp, A, B, n_rows, n_cols, P, value_type, mode):
    dA = crp.to_device(A)
    dB = dA if B is A else crp.to_device(B)
    plan = crp.Plan(n_rows, n_cols, P, ci.SEED_A, ci.SEED_B, value_type=value_type, mode=mode)
    plan.accumulate(dA, dB)
    plan.sync()
    i, j, w, _ = plan.export()
    plan.close()
    return i, j, w


def _sorted(i, j, w):
    o = np.lexsort((j, i))
    return i[o], j[o], w[o]


def _real_case():
    rng = np.random.default_rng(7)
    K, n = 400, 300
    ptrs, idxs = [], []
    for _ in range(2):
        L = rng.integers(0, 25, K)
        ptrs.append(np.concatenate([[0], np.cumsum(L)]).astype(np.int64))
        idxs.append(np.concatenate([np.sort(rng.choice(n, l, replace=False)) for l in L]
                                   ).astype(np.int32))
    A = ci.Sparse(ptrs[0], idxs[0], rng.uniform(0.01, 2, len(idxs[0])).astype(np.float32), n)
    B = ci.Sparse(ptrs[1], idxs[1], rng.uniform(0.01, 2, len(idxs[1])).astype(np.float32), n)
    return A, B


def test_noalloc_matches_plan_path_on_consecutive_calls(crp):
    T = ci.C1.generate()
    A, B = _real_case()
    cases = [
        (T, T, 1000, 1000, 64, crp.CRP_I32, crp.CRP_FULL),
        (A, B, 300, 300, 16, crp.CRP_F32_COMP, crp.CRP_UPPER),
        (T, T, 1000, 1000, 256, crp.CRP_I32, crp.CRP_UPPER),
    ]
    for (X, Y, nr, nc, P, vt, mode) in cases:
        want = _sorted(*_with_plan(crp, X, Y, nr, nc, P, vt, mode))
        got = _sorted(*_noalloc(crp, X, Y, nr, nc, P, vt, mode, capacity=len(want[0]) + 10))
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        if vt == crp.CRP_I32:
            assert np.array_equal(got[2], want[2])
        else:
            np.testing.assert_allclose(got[2], want[2], rtol=RTOL_REAL, atol=0)


def test_noalloc_rejects_sizes_beyond_its_limits(crp):
    T = ci.C1.scaled(m=100).generate()
    d = crp.crp_plan_desc()
    d.n_rows = d.n_cols = 1000
    d.P = 2048                      # more partitions than the static table holds
    dT = crp.to_device(T)
    a = dT.c_struct()
    n = ctypes.c_int64(0)
    st = crp.lib().crp_outer_product_noalloc(ctypes.byref(d), ctypes.byref(a), ctypes.byref(a),
                                             None, None, None, 0, ctypes.byref(n), None)
    assert st == crp.CRP_EINVAL
    assert b"1024" in crp.lib().crp_last_error()


def _raw_call(crp, desc, a, b, i, j, w, capacity):
    """One call of the entry point on prepared device buffers; returns the
    status and *n_out."""
    import torch
    n = ctypes.c_int64(-1)
    stream = torch.cuda.current_stream().cuda_stream
    st = crp.lib().crp_outer_product_noalloc(
        ctypes.byref(desc), ctypes.byref(a), ctypes.byref(b),
        i.data_ptr() if i is not None else None, j.data_ptr() if j is not None else None,
        w.data_ptr() if w is not None else None, capacity, ctypes.byref(n), stream)
    return st, n.value


def _desc(crp, n_rows, n_cols, P, value_type=0, mode=0):
    d = crp.crp_plan_desc()
    d.n_rows, d.n_cols, d.P = n_rows, n_cols, P
    d.seed_a, d.seed_b = ci.SEED_A, ci.SEED_B
    d.value_type, d.mode = value_type, mode
    return d


def test_noalloc_allocates_nothing_and_handles_one_partition(crp):
    """The point of the entry point: a call moves neither the device's free
    memory (cudaMemGetInfo) nor PyTorch's allocator.  The second and third
    calls are measured (the first may load the library's kernels).  P = 1 puts
    every entry into one partition of 2^20 slots."""
    import torch
    T = ci.C1.generate()
    want = _sorted(*_with_plan(crp, T, T, 1000, 1000, 1, crp.CRP_I32, crp.CRP_FULL))
    dT = crp.to_device(T)
    a = dT.c_struct()
    cap = len(want[0]) + 5
    i = torch.empty(cap, dtype=torch.int32, device="cuda")
    j = torch.empty(cap, dtype=torch.int32, device="cuda")
    w = torch.empty(cap, dtype=torch.float64, device="cuda")
    d = _desc(crp, 1000, 1000, 1)
    st, n = _raw_call(crp, d, a, a, i, j, w, cap)
    assert st == crp.CRP_OK, crp.lib().crp_last_error()
    torch.cuda.synchronize()
    for _ in range(2):
        free0, _ = torch.cuda.mem_get_info()
        stats0 = torch.cuda.memory_stats()
        st, n = _raw_call(crp, d, a, a, i, j, w, cap)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        stats1 = torch.cuda.memory_stats()
        assert st == crp.CRP_OK, crp.lib().crp_last_error()
        assert free1 == free0
        for key in ("allocation.all.allocated", "segment.all.allocated"):
            assert stats1.get(key, 0) == stats0.get(key, 0), key
        assert n == len(want[0])
        got = _sorted(i[:n].cpu().numpy(), j[:n].cpu().numpy(), w[:n].cpu().numpy())
        for g, x in zip(got, want):
            assert np.array_equal(g, x)


def test_noalloc_short_output_reports_the_size_needed(crp):
    """capacity below the entry count: CRP_EINVAL, *n_out = the number of
    entries the plan path finds, and nothing written past the capacity."""
    import torch
    T = ci.C1.generate()
    want = _with_plan(crp, T, T, 1000, 1000, 64, crp.CRP_I32, crp.CRP_FULL)
    dT = crp.to_device(T)
    a = dT.c_struct()
    i = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    j = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    w = torch.full((4,), -7.0, dtype=torch.float64, device="cuda")
    st, n = _raw_call(crp, _desc(crp, 1000, 1000, 64), a, a, i, j, w, 1)
    assert st == crp.CRP_EINVAL
    assert n == len(want[0])
    assert (i[1:].cpu().numpy() == -7).all() and (j[1:].cpu().numpy() == -7).all()
    assert (w[1:].cpu().numpy() == -7.0).all()


def test_noalloc_reports_a_full_partition_and_recovers(crp):
    """A product with more entries than a partition of the static table holds
    (100,000 transactions of the 10M-transaction recipe, P = 1024: ~1,000
    slots per partition, ~10^4 entries per partition) returns
    CRP_ETABLE_FULL with *n_out = 0; the next call, on a product that fits,
    is exact again (the full marks are cleared)."""
    import torch
    big = ci.C2.scaled(m=100_000).generate()
    dB = crp.to_device(big)
    b = dB.c_struct()
    cap = 1 << 20
    i = torch.empty(cap, dtype=torch.int32, device="cuda")
    j = torch.empty(cap, dtype=torch.int32, device="cuda")
    w = torch.empty(cap, dtype=torch.float64, device="cuda")
    st, n = _raw_call(crp, _desc(crp, big.n_minor, big.n_minor, 1024), b, b, i, j, w, cap)
    assert st == crp.CRP_ETABLE_FULL
    assert n == 0
    assert b"static table" in crp.lib().crp_last_error()
    T = ci.C1.generate()
    want = _sorted(*_with_plan(crp, T, T, 1000, 1000, 64, crp.CRP_I32, crp.CRP_UPPER))
    got = _sorted(*_noalloc(crp, T, T, 1000, 1000, 64, crp.CRP_I32, crp.CRP_UPPER,
                            capacity=len(want[0])))
    for g, x in zip(got, want):
        assert np.array_equal(g, x)
