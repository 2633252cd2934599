"""The entry point that allocates no device memory (dfpr_static_pagerank_noalloc),
called through the C ABI and checked against the CPU oracle's reference ranks
and against the library's own dfpr_static_pagerank (Jacobi schedule) on the
same graphs, within the FP64 tolerance of the other tests.

It serves callers that cannot call cudaMalloc / cudaFree (a framework or
server that owns the whole device memory budget, or code that must not cause
the synchronisation those calls imply); its scratch is a fixed device array
shared by every call. This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9
MAX_VERTICES = 1 << 20


def device_graph(dfpr, torch, n, src, dst, dead_end=0):
    """In-rows, out-degrees (device tensors) and the library's own static ranks."""
    g = dfpr.graph_load(n, src, dst, dfpr.default_config(dead_end=dead_end))
    m = g.info()["m"]
    in_off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    in_idx = torch.empty(m, dtype=torch.int32, device="cuda")
    g.get_csc(in_off, in_idx)
    out_off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    out_idx = torch.empty(m, dtype=torch.int32, device="cuda")
    g.get_csr(out_off, out_idx)
    out_deg = (out_off[1:] - out_off[:-1]).to(torch.int32).contiguous()
    st = g.static_pagerank(dfpr.default_params(mode=dfpr.JACOBI))
    assert st.status == dfpr.OK
    lib_ranks = g.get_ranks()
    torch.cuda.synchronize()
    return g, in_off, in_idx, out_deg, lib_ranks, st.passes


def call_noalloc(lib, n, in_off, in_idx, out_deg, ranks, tol=1e-10, max_iter=500):
    it = ctypes.c_int32(-1)
    rc = lib.dfpr_static_pagerank_noalloc(n, in_off.data_ptr(), in_idx.data_ptr(),
                                          out_deg.data_ptr(), 0.85, tol, max_iter,
                                          ranks.data_ptr(), ctypes.byref(it), None)
    return rc, it.value


def test_noalloc_matches_oracle_and_static_pagerank_twice(gpu_lib):
    import torch
    lib = gpu_lib.load()
    # self-loops (the paper's graphs), and a teleport graph whose dead ends
    # spread their rank uniformly
    cases = [(workloads.rmat_graph(14, 16, 1), gpu_lib.SELF_LOOPS),
             (workloads.rmat_graph(12, 8, 7), gpu_lib.SELF_LOOPS),
             (workloads.rmat_graph(12, 4, 9), gpu_lib.TELEPORT)]
    prepared, expect = [], []
    for (n, s, d), de in cases:
        prepared.append(device_graph(gpu_lib, torch, n, s, d, de))
        ref, _ = oracle.Graph.build(n, s, d, self_loops=(de == gpu_lib.SELF_LOOPS)).reference(dead_end=de)
        expect.append(ref)
    n_dead = int((prepared[2][3] == 0).sum().item())
    assert n_dead > 0  # the teleport case has dead ends
    # calls in a row on different graphs, then the first graph again: the
    # shared scratch keeps the previous call's contents and must not leak
    for k in (0, 1, 2, 0, 2):
        n = cases[k][0][0]
        _, in_off, in_idx, out_deg, lib_ranks, passes = prepared[k]
        ranks = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc, iters = call_noalloc(lib, n, in_off, in_idx, out_deg, ranks)
        assert rc == gpu_lib.OK, gpu_lib.last_error()
        assert abs(iters - passes) <= 1  # summation order differs at the stopping boundary
        got = ranks.cpu().numpy()
        assert float(np.max(np.abs(got - expect[k]))) <= LINF64
        assert float(np.max(np.abs(got - lib_ranks))) <= LINF64
        assert abs(float(got.sum()) - 1.0) < 1e-9  # no rank leaks through dead ends


def test_noalloc_iteration_cap_returns_the_last_iterate(gpu_lib):
    # an odd and an even cap: the last iterate sits in the scratch vector or
    # in the caller's buffer, and must reach the caller either way
    import torch
    lib = gpu_lib.load()
    n, s, d = workloads.rmat_graph(11, 8, 5)
    _, in_off, in_idx, out_deg, _, _ = device_graph(gpu_lib, torch, n, s, d)
    g0 = oracle.Graph.build(n, s, d)
    for cap in (3, 4):
        ranks = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc, iters = call_noalloc(lib, n, in_off, in_idx, out_deg, ranks, tol=1e-300, max_iter=cap)
        assert rc == gpu_lib.ENOTCONV and iters == cap
        want, st = g0.static_bb(tol=1e-300, max_iter=cap)   # the cap-th Jacobi iterate
        assert st.iterations == cap and not st.converged
        assert float(np.max(np.abs(ranks.cpu().numpy() - want))) <= 1e-15


def test_noalloc_allocates_nothing(gpu_lib):
    # after the first call on the device (which may load the library's module),
    # a call changes neither the device's free memory nor calls the library's
    # allocator hook
    import torch
    lib = gpu_lib.load()
    n, s, d = workloads.rmat_graph(12, 8, 3)
    g, in_off, in_idx, out_deg, lib_ranks, _ = device_graph(gpu_lib, torch, n, s, d)
    ranks = torch.empty(n, dtype=torch.float64, device="cuda")
    rc, _ = call_noalloc(lib, n, in_off, in_idx, out_deg, ranks)
    assert rc == gpu_lib.OK
    torch.cuda.synchronize()
    calls = []

    def counting_alloc(nbytes, stream):
        calls.append(nbytes)
        return 0  # refuse: any allocation would fail the call

    def counting_free(ptr, nbytes, stream):
        calls.append(-1)

    gpu_lib.set_allocator(counting_alloc, counting_free)
    try:
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            rc, _ = call_noalloc(lib, n, in_off, in_idx, out_deg, ranks)
            assert rc == gpu_lib.OK, gpu_lib.last_error()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        gpu_lib.set_allocator(None, None)
    assert calls == []
    assert free1 == free0
    assert float(np.max(np.abs(ranks.cpu().numpy() - lib_ranks))) <= LINF64


def test_noalloc_rejects_sizes_beyond_the_scratch(gpu_lib):
    import torch
    lib = gpu_lib.load()
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = lib.dfpr_static_pagerank_noalloc(MAX_VERTICES + 1, dummy.data_ptr(), dummy.data_ptr(),
                                          dummy.data_ptr(), 0.85, 1e-10, 500, dummy.data_ptr(),
                                          None, None)
    assert rc == gpu_lib.EINVAL
    assert "exceeds" in gpu_lib.last_error()
