"""dfpr_autotune and the degree-class thresholds (gather_split, mark_split):
the tuner times the same pending update under each candidate, applies it once
with the fastest, and the result is the oracle's within the usual bound."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9


@pytest.fixture(scope="module")
def case():
    n, src, dst = workloads.rmat_graph(14, 16, 31)
    batch = workloads.uniform_batch(n, 1000, 32, src, dst)
    g0 = oracle.Graph.build(n, src, dst)
    g1, _ = g0.apply(*batch)
    R0, _ = g0.reference()
    ref1, _ = g1.reference()
    return dict(n=n, src=src, dst=dst, batch=batch, R0=R0, ref1=ref1)


def updated(gpu_lib, case):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    g.set_ranks(case["R0"])
    g.apply_batch(*case["batch"])
    return g


def test_default_candidates(gpu_lib, case):
    g = updated(gpu_lib, case)
    p, trials, st = g.autotune()
    assert st.status == gpu_lib.OK
    assert (p.gather_split, p.mark_split) in [(2048, 2048), (4096, 8192), (8192, 8192), (16384, 16384)]
    assert trials.shape == (4,) and np.all(np.isfinite(trials)) and np.all(trials > 0)
    assert trials[[(2048, 2048), (4096, 8192), (8192, 8192), (16384, 16384)].index(
        (p.gather_split, p.mark_split))] == trials.min()
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64
    # the pending change set was consumed once, by the final update
    assert g.df_pagerank().processed == 0


def test_custom_candidates_and_errors(gpu_lib, case):
    g = updated(gpu_lib, case)
    p, trials, st = g.autotune(candidates=[(256, 256), (1024, 4096)])
    assert st.status == gpu_lib.OK and len(trials) == 2
    assert (p.gather_split, p.mark_split) in [(256, 256), (1024, 4096)]
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64
    with pytest.raises(gpu_lib.DfprError) as e:  # nothing pending now
        g.autotune()
    assert e.value.status == gpu_lib.EINVAL
    g2 = updated(gpu_lib, case)
    for bad in ([(100, 4096)], [(4096, 1 << 25)]):
        with pytest.raises(gpu_lib.DfprError) as e:
            g2.autotune(candidates=bad)
        assert e.value.status == gpu_lib.EINVAL
    with pytest.raises(gpu_lib.DfprError) as e:
        g2.autotune(gpu_lib.default_params(mode=gpu_lib.JACOBI))
    assert e.value.status == gpu_lib.EINVAL
    assert g2.df_pagerank().status == gpu_lib.OK  # still pending after the refusals
    assert np.max(np.abs(g2.get_ranks() - case["ref1"])) <= LINF64


@pytest.mark.parametrize("mode", ["WORKLIST", "ROUND"])
def test_thresholds_decide_the_split(gpu_lib, case, mode):
    """A low gather_split cuts the hubs' in-rows into tokens; the largest
    allowed one leaves every row to a single warp. Both give the same ranks."""
    out = {}
    for gs in (256, 1 << 24):
        g = updated(gpu_lib, case)
        st = g.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode), gather_split=gs,
                                                  mark_split=gs))
        assert st.status == gpu_lib.OK
        assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64
        out[gs] = st
    if mode == "WORKLIST":
        assert out[256].jobs > 0 and out[256].tokens > 0
        assert out[1 << 24].jobs == 0 and out[1 << 24].tokens == 0


def test_plans_cover_schedules_and_size_classes(gpu_lib, case):
    g = updated(gpu_lib, case)
    p, plans, trials, st = g.autotune_plans()
    assert st.status == gpu_lib.OK
    modes = set(plans[:, 0].tolist())
    assert gpu_lib.WORKLIST in modes and gpu_lib.JACOBI in modes
    assert len({int(x) for x in plans[plans[:, 0] == gpu_lib.WORKLIST, 1]}) >= 2   # grid sizes
    assert np.all(np.isfinite(trials)) and np.all(trials > 0)
    best = int(np.argmin(trials))
    assert (p.mode, p.grid_ctas, p.gather_split, p.mark_split) == tuple(int(x) for x in plans[best])
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64
    assert g.df_pagerank().processed == 0   # the pending set was consumed once


def test_explicit_plans(gpu_lib, case):
    g = updated(gpu_lib, case)
    p, plans, trials, st = g.autotune_plans(plans=[(gpu_lib.JACOBI, 0, 0, 0)])
    assert st.status == gpu_lib.OK and p.mode == gpu_lib.JACOBI and len(trials) == 1
    assert np.max(np.abs(g.get_ranks() - case["ref1"])) <= LINF64
    g2 = updated(gpu_lib, case)
    p, plans, trials, st = g2.autotune_plans(plans=[(gpu_lib.WORKLIST, 16, 0, 0),
                                                    (gpu_lib.ROUND, 0, 4096, 8192)])
    assert st.status == gpu_lib.OK and len(trials) == 2
    assert np.max(np.abs(g2.get_ranks() - case["ref1"])) <= LINF64
    with pytest.raises(gpu_lib.DfprError) as e:
        g2.autotune_plans(plans=[(gpu_lib.WORKLIST, 0, 0, 0)])   # nothing pending
    assert e.value.status == gpu_lib.EINVAL
