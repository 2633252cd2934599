"""Termination of the worklist schedule.

(1) FP32 ranks on a near-uniform grid, where most ranks sit just above a
    power of two and one ulp is above the relative tolerance: FP32 evaluates
    Eq. 1 with each vertex's current rank in its self-loop term, which damps
    rounding jitter (solving that term in closed form, as FP64 does, let
    neighbours flip each other by an ulp or two for ever). The updates end,
    with bounded work, at an FP32-sized residual of Eq. 1.
(2) The stop conditions (the work cap of max_iter * n recomputations, the time
    budget) end a launch whose queue never drains: a static worklist run from
    1/n capped at 2n recomputations stops within one poll interval per warp of
    the cap instead of running to convergence."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [256, 1024])
def test_fp32_grid_updates_terminate(gpu_lib, L):
    dfpr = gpu_lib
    n, src, dst = workloads.grid_graph(L, 4)
    g = dfpr.graph_load(n, src, dst, dfpr.default_config(precision=dfpr.FP32))
    m0 = g.info()["m"]
    # Jacobi below the FP32 resolution stops at the cap, at a float fixed point
    # of the synchronous iteration
    st = dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, tol=1e-10, max_iter=300))
    assert st.status in (dfpr.OK, dfpr.ENOTCONV)
    b = max(1, int(round(1e-4 * m0)))
    for i in range(3):
        dfpr.apply_batch(g, *workloads.grid_local_batch(L, b, 300 + i))
        st = dfpr.df_pagerank(g, dfpr.default_params(tol=1e-7, timeout_ms=5000))
        # the work cap is 500 n; the first update also moves the ranks from
        # the synchronous iteration's float state to the asynchronous one
        assert st.status == dfpr.OK
        assert st.processed < (100 if i == 0 else 4) * n
        _, rel = dfpr.residual(g)
        assert rel <= 5e-7  # a few FP32 ulps of Eq. 1
    g.free()


def test_work_cap_ends_a_busy_queue(gpu_lib):
    dfpr = gpu_lib
    n, src, dst = workloads.rmat_graph(16, 16, 21)
    g = dfpr.graph_load(n, src, dst)
    grid = 2
    warps = grid * 8  # 256 threads per block
    st = dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.WORKLIST, max_iter=2,
                                                     grid_ctas=grid))
    assert st.status == dfpr.ENOTCONV
    cap = 2 * n
    # each warp adds its local count (< 2048) to the total, then polls the
    # stop flag at most 16 batches of 32 vertices later
    slack = warps * (2048 + 17 * 32)
    assert cap < st.processed <= cap + slack
    # a full run from 1/n takes many more recomputations than the cap
    full = dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.WORKLIST, grid_ctas=grid))
    assert full.status == dfpr.OK and full.processed > cap + slack
    g.free()
