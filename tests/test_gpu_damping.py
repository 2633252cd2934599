"""Damping factors other than the paper's 0.85. Eq. 1 holds for any alpha in
(0, 1), and the library takes alpha as a parameter. Checked here:
- static and DF updates on every schedule, against the oracle's reference
  at the same alpha;
- the jacobi DF against the oracle's DF_BB (Alg. 1), iteration by
  iteration.

Bound: a schedule stops once the ranks move by at most tol per step, and a
geometric tail after that adds at most tol * alpha / (1 - alpha). Twice that
is allowed, since the asynchronous schedules judge each vertex by its own
change. At alpha = 0.95 the reference after 500 iterations is within
alpha^500 of the fixed point, about 7e-12 relative.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10
MODES = ["WORKLIST", "ROUND", "JACOBI"]
# The paper's MAX_ITERATIONS = 500 is set for alpha = 0.85. An iteration
# shrinks the error by about alpha, so alpha = 0.95 needs about
# log(0.85) / log(0.95) = 3.2 times the passes. The round schedule's
# lock-free passes came within reach of 500 there, so the cap is scaled.
MAX_ITER = 2000


def bound(alpha):
    return 2.0 * TOL * alpha / (1.0 - alpha) + 1e-13


@pytest.fixture(scope="module", params=[0.5, 0.95])
def case(request):
    alpha = request.param
    n, src, dst = workloads.rmat_graph(14, 16, 1)
    batch = workloads.uniform_batch(n, 1000, 2, src, dst)
    g0 = oracle.Graph.build(n, src, dst)
    g1, nreal = g0.apply(*batch)
    ref0, _ = g0.static_bb(alpha=alpha, tol=oracle.REF_TOL, max_iter=oracle.MAX_ITER)
    ref1, _ = g1.static_bb(alpha=alpha, tol=oracle.REF_TOL, max_iter=oracle.MAX_ITER)
    return dict(alpha=alpha, n=n, src=src, dst=dst, batch=batch, g1=g1, nreal=nreal,
                ref0=ref0, ref1=ref1)


@pytest.mark.parametrize("mode", MODES)
def test_static_at_other_damping(gpu_lib, case, mode):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    st = g.static_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode), alpha=case["alpha"],
                                                  tol=TOL, max_iter=MAX_ITER))
    assert st.status == gpu_lib.OK
    err = np.max(np.abs(g.get_ranks() - case["ref0"]))
    assert err <= bound(case["alpha"]), err


@pytest.mark.parametrize("mode", MODES)
def test_df_at_other_damping(gpu_lib, case, mode):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    g.set_ranks(case["ref0"])
    assert g.apply_batch(*case["batch"]) == case["nreal"]
    st = g.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode), alpha=case["alpha"],
                                              tol=TOL, max_iter=MAX_ITER))
    assert st.status == gpu_lib.OK, st.as_dict()
    err = np.max(np.abs(g.get_ranks() - case["ref1"]))
    assert err <= bound(case["alpha"]), err


def test_jacobi_df_follows_oracle_df_bb(gpu_lib, case):
    g = gpu_lib.graph_load(case["n"], case["src"], case["dst"])
    g.set_ranks(case["ref0"])
    g.apply_batch(*case["batch"])
    st = g.df_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI, alpha=case["alpha"], tol=TOL,
                                              max_iter=MAX_ITER))
    R_o, st_o = case["g1"].df_bb(case["ref0"], alpha=case["alpha"], tol=TOL, max_iter=MAX_ITER)
    assert st.passes == st_o.iterations
    assert st.affected == st_o.affected
    assert np.max(np.abs(g.get_ranks() - R_o)) <= 1e-12
