"""The entry point that allocates no device memory (dfpr_static_pagerank_noalloc),
called through the C ABI and checked against dfpr_static_pagerank (Jacobi
schedule) on the same graphs, within the FP64 tolerance of the other tests.

It serves callers that cannot call cudaMalloc / cudaFree (a framework or
server that owns the whole device memory budget, or code that must not cause
the synchronisation those calls imply); its scratch is a fixed device array
shared by every call. This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9
MAX_VERTICES = 1 << 20


def device_graph(dfpr, torch, n, src, dst):
    """In-rows, out-degrees (device tensors) and the library's own static ranks."""
    g = dfpr.graph_load(n, src, dst)
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
    ref = g.get_ranks()
    torch.cuda.synchronize()
    return in_off, in_idx, out_deg, ref, st.passes


def call_noalloc(lib, n, in_off, in_idx, out_deg, ranks, tol=1e-10, max_iter=500):
    it = ctypes.c_int32(-1)
    rc = lib.dfpr_static_pagerank_noalloc(n, in_off.data_ptr(), in_idx.data_ptr(),
                                          out_deg.data_ptr(), 0.85, tol, max_iter,
                                          ranks.data_ptr(), ctypes.byref(it), None)
    return rc, it.value


def test_noalloc_matches_static_pagerank_twice(gpu_lib):
    import torch
    lib = gpu_lib.load()
    graphs = [workloads.rmat_graph(14, 16, 1), workloads.rmat_graph(12, 8, 7)]
    prepared = [device_graph(gpu_lib, torch, n, s, d) for n, s, d in graphs]
    # two calls in a row on different graphs, then the first graph again: the
    # shared scratch keeps the previous call's contents and must not leak
    for k in (0, 1, 0):
        n = graphs[k][0]
        in_off, in_idx, out_deg, ref, passes = prepared[k]
        ranks = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc, iters = call_noalloc(lib, n, in_off, in_idx, out_deg, ranks)
        assert rc == gpu_lib.OK, gpu_lib.last_error()
        assert abs(iters - passes) <= 1  # summation order differs at the stopping boundary
        err = float(np.max(np.abs(ranks.cpu().numpy() - ref)))
        assert err <= LINF64, err


def test_noalloc_rejects_sizes_beyond_the_scratch(gpu_lib):
    import torch
    lib = gpu_lib.load()
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = lib.dfpr_static_pagerank_noalloc(MAX_VERTICES + 1, dummy.data_ptr(), dummy.data_ptr(),
                                          dummy.data_ptr(), 0.85, 1e-10, 500, dummy.data_ptr(),
                                          None, None)
    assert rc == gpu_lib.EINVAL
    assert "exceeds" in gpu_lib.last_error()
