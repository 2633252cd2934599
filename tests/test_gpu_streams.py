"""Device memory from torch's caching allocator, and a graph moved between
streams. A stream the library created stays alive until the graph is freed,
because arrays allocated on it name it when they are released. Results match
the oracle on every stream, and every byte returns to torch's pool."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9


def test_torch_allocator_and_stream_switches(gpu_lib):
    import torch
    n, src, dst = workloads.rmat_graph(14, 16, 1)
    batch = workloads.uniform_batch(n, 1000, 2, src, dst)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.reference()
    g1, nreal = g0.apply(*batch)
    ref1, _ = g1.reference()

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    gpu_lib.use_torch_allocator()
    try:
        g = gpu_lib.graph_load(n, src, dst, stream=None)  # on a stream of the library's
        assert torch.cuda.memory_allocated() > before    # the graph lives in torch's pool
        g.set_ranks(R0)
        side = torch.cuda.Stream()
        gpu_lib.graph_set_stream(g, side.cuda_stream)     # the library's stream is retired
        assert g.apply_batch(*batch) == nreal
        st = g.df_pagerank(gpu_lib.default_params())
        assert st.status == gpu_lib.OK
        assert np.max(np.abs(g.get_ranks() - ref1)) <= LINF64
        gpu_lib.graph_set_stream(g, None)                 # a new stream of the library's
        st = g.static_pagerank(gpu_lib.default_params())
        assert st.status == gpu_lib.OK
        assert np.max(np.abs(g.get_ranks() - ref1)) <= LINF64
        g.free()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before    # every array went back
    finally:
        gpu_lib.set_allocator(None, None)
