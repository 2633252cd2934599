"""dfpr_get_ranks into every kind of destination: device memory, page-locked
host memory (written by the device directly) and pageable host memory
(through the graph's staging vector). All three give the same bits, in the
caller's vertex numbering, for FP64 and FP32 graphs."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_get_ranks_destinations_agree(gpu_lib, prec):
    import torch
    dfpr = gpu_lib
    n, src, dst = workloads.rmat_graph(14, 16, 3)
    g = dfpr.graph_load(n, src, dst, dfpr.default_config(precision=getattr(dfpr, prec)))
    assert dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI,
                                                       tol=1e-12 if prec == "FP64" else 1e-7)).status == dfpr.OK
    pageable = dfpr.get_ranks(g)
    pinned = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
    dfpr.get_ranks(g, pinned)
    dev = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    dfpr.get_ranks(g, dev)
    assert np.array_equal(pageable, pinned.numpy())
    assert np.array_equal(pageable, dev.cpu().numpy())
    assert np.all(pageable > 0) and abs(pageable.sum() - 1.0) < 1e-5
    # a second pageable read reuses the staging vector; the ranks round-trip
    dfpr.set_ranks(g, pageable[::-1].copy())
    assert np.array_equal(dfpr.get_ranks(g), pageable[::-1])
    g.free()
