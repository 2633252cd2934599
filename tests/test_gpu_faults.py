"""Simulated thread delays and crash-stops (Sec. 5.1.6, 5.3, 5.4) on the GPU.

A warp stands for one of the paper's threads. Delays are bounded sleeps after
a batch of vertices; a crash-stop is a warp that returns at a random batch
boundary without finishing its bookkeeping. Nothing here faults or hangs the
GPU: every wait in the kernels is bounded by the call's time budget.

Expected behaviour, as in the paper: the lock-free schedules finish with the
same accuracy despite delays and crashes. The round schedule (Alg. 2) does so
through its passes and R_C flags; the worklist schedule through helping (Sec.
4.4): idle warps return the claimed vertices of a warp that stopped to the
queue. With helping off, a crashed worklist warp leaves the count of open work
unbalanced, so the call stops at the time budget (a bounded wait that runs
out). The barrier-based jacobi schedule tolerates delays but cannot complete
with a crashed thread (it rejects the request).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9
GRID = 8           # CTAs of the launch: 64 warps (the round schedule's own limit here)
WARPS = GRID * 8


@pytest.fixture(scope="module")
def case():
    n, src, dst = workloads.rmat_graph(14, 16, 1)
    batch = workloads.uniform_batch(n, 1000, 2, src, dst)
    g0 = oracle.Graph.build(n, src, dst)
    g1, _ = g0.apply(*batch)
    R0, _ = g0.reference()
    ref0 = R0
    ref1, _ = g1.reference()
    return dict(n=n, src=src, dst=dst, batch=batch, R0=R0, ref0=ref0, ref1=ref1)


def updated_graph(gpu_lib, case):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    g.set_ranks(case["R0"])
    g.apply_batch(*case["batch"])
    return g


def params(gpu_lib, mode, **kw):
    return gpu_lib.default_params(mode=getattr(gpu_lib, mode), grid_ctas=GRID, **kw)


@pytest.mark.parametrize("crashed", [1, WARPS // 2, WARPS - 1])
def test_round_schedule_finishes_despite_crashes(gpu_lib, case, crashed):
    g = updated_graph(gpu_lib, case)
    st = g.df_pagerank(params(gpu_lib, "ROUND", fault_crash_warps=crashed, fault_seed=7))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64


def test_round_static_finishes_despite_crashes(gpu_lib, case):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    st = g.static_pagerank(params(gpu_lib, "ROUND", fault_crash_warps=WARPS // 2, fault_seed=3))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref0"])) <= LINF64


@pytest.mark.parametrize("mode", ["ROUND", "WORKLIST", "JACOBI"])
def test_delays_keep_accuracy(gpu_lib, case, mode):
    g = updated_graph(gpu_lib, case)
    st = g.df_pagerank(params(gpu_lib, mode, fault_delay_prob=2e-3, fault_delay_us=300.0,
                              fault_seed=11))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64
    assert st.ms >= 0.3  # at least one 300-us sleep happened


@pytest.mark.parametrize("crashed", [1, WARPS // 2, WARPS - 1])
def test_worklist_finishes_despite_crashes(gpu_lib, case, crashed):
    """Helping: the vertices a crashed warp held go back to the queue."""
    g = updated_graph(gpu_lib, case)
    st = g.df_pagerank(params(gpu_lib, "WORKLIST", fault_crash_warps=crashed, fault_seed=5))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64


def test_worklist_static_finishes_despite_crashes(gpu_lib, case):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    st = g.static_pagerank(params(gpu_lib, "WORKLIST", fault_crash_warps=WARPS // 2, fault_seed=3))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref0"])) <= LINF64


def test_worklist_crash_without_helping_stops_at_the_time_budget_and_recovers(gpu_lib, case):
    g = updated_graph(gpu_lib, case)
    st = g.df_pagerank(params(gpu_lib, "WORKLIST", fault_crash_warps=WARPS // 2, fault_seed=5,
                              timeout_ms=300.0, helping=0))
    assert st.status == gpu_lib.ETIMEOUT
    st = g.nd_pagerank(gpu_lib.default_params())  # the graph stays usable
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64


def test_jacobi_rejects_crashes_and_bad_fault_parameters(gpu_lib, case):
    g = updated_graph(gpu_lib, case)
    bad = [dict(mode="JACOBI", fault_crash_warps=1),
           dict(mode="ROUND", fault_delay_prob=1.5),
           dict(mode="ROUND", fault_delay_us=2e6),
           dict(mode="ROUND", fault_crash_warps=-1),
           dict(mode="ROUND", fault_crash_warps=WARPS),  # every warp of the launch
           dict(mode="WORKLIST", helping=2)]
    for kw in bad:
        mode = kw.pop("mode")
        with pytest.raises(gpu_lib.DfprError) as e:
            g.df_pagerank(params(gpu_lib, mode, **kw))
        assert e.value.status == gpu_lib.EINVAL, kw
    st = g.df_pagerank(params(gpu_lib, "ROUND"))  # still pending, still correct
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64


def test_same_seed_same_crashing_warps(gpu_lib, case):
    """The draws are counter-based: a seed fixes which warps crash."""
    out = []
    for _ in range(2):
        g = updated_graph(gpu_lib, case)
        st = g.df_pagerank(params(gpu_lib, "WORKLIST", fault_crash_warps=WARPS - 1, fault_seed=9,
                                  timeout_ms=200.0, helping=0))
        out.append(st.status)
    assert out == [gpu_lib.ETIMEOUT, gpu_lib.ETIMEOUT]
