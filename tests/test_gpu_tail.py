"""The FP64 tail of the precision split: the final normalisation (normalize = 1,
an FP64 sum of the ranks and a rescale) and the FP64 residual of Eq. 1 over
all vertices (dfpr_residual), on both precisions. The residual is checked
against a numpy evaluation of Eq. 1 on the exported graph and ranks."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def numpy_residual(dfpr, g, alpha=0.85, teleport=False):
    """max_v |Eq. 1 (v) - R[v]| and the same relative to R[v], in FP64 from the
    exported CSR, CSC and ranks (numpy only)."""
    n = g.n
    R = dfpr.get_ranks(g)
    out_off, _ = dfpr.get_csr(g)
    in_off, in_idx = dfpr.get_csc(g)
    outdeg = np.diff(out_off).astype(np.float64)
    contrib = np.where(outdeg > 0, R / np.maximum(outdeg, 1), 0.0)
    s = np.zeros(n)
    has = np.diff(in_off) > 0
    sums = np.add.reduceat(contrib[in_idx], in_off[:-1][has]) if has.any() else np.zeros(0)
    s[has] = sums
    dead = R[outdeg == 0].sum() if teleport else 0.0
    r = (1 - alpha) / n + alpha * (s + dead / n)
    res = np.abs(r - R)
    return res.max(), (res / R).max()


@pytest.mark.parametrize("prec,dead_end", [("FP64", "SELF_LOOPS"), ("FP32", "SELF_LOOPS"),
                                            ("FP64", "TELEPORT")])
def test_residual_matches_numpy(gpu_lib, prec, dead_end):
    dfpr = gpu_lib
    n, src, dst = workloads.rmat_graph(12, 8, 4)
    g = dfpr.graph_load(n, src, dst, dfpr.default_config(precision=getattr(dfpr, prec),
                                                         dead_end=getattr(dfpr, dead_end)))
    # a few Jacobi iterations from 1/n: far from converged, so the residual is large
    st = dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, max_iter=4))
    assert st.status == dfpr.ENOTCONV
    linf, rel = dfpr.residual(g)
    want, want_rel = numpy_residual(dfpr, g, teleport=dead_end == "TELEPORT")
    assert want > 1e-6
    assert abs(linf - want) <= 1e-12 * want + 1e-18
    assert abs(rel - want_rel) <= 1e-10 * want_rel
    g.free()


def test_residual_after_df_update_is_small(gpu_lib):
    dfpr = gpu_lib
    n, src, dst = workloads.rmat_graph(14, 16, 1)
    batch = workloads.uniform_batch(n, 1000, 2, src, dst)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.reference()
    g1, _ = g0.apply(*batch)
    ref, _ = g1.reference()
    g = dfpr.graph_load(n, src, dst)
    dfpr.set_ranks(g, R0)
    dfpr.apply_batch(g, *batch)
    st = dfpr.df_pagerank(g)
    assert st.status == dfpr.OK
    linf, _ = dfpr.residual(g)
    assert linf <= 1e-10          # at the iteration tolerance tau
    assert float(np.max(np.abs(dfpr.get_ranks(g) - ref))) <= 1e-9
    # the reference itself is a fixed point of Eq. 1 to FP64 rounding
    dfpr.set_ranks(g, ref)
    assert dfpr.residual(g)[0] <= 1e-15
    g.free()


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_normalize_rescales_to_sum_one(gpu_lib, prec):
    # Two copies of a graph start from the same ranks, scaled by 1.25 so that
    # they do not sum to 1, take the same batch and the same deterministic
    # (Jacobi) DF update; one with normalize = 1. Its ranks must be the other's
    # divided by their FP64 sum, and its reported rank_sum 1.
    dfpr = gpu_lib
    P = getattr(dfpr, prec)
    tol = 1e-10 if prec == "FP64" else 1e-7
    n, src, dst = workloads.rmat_graph(13, 16, 6)
    a = dfpr.graph_load(n, src, dst, dfpr.default_config(precision=P))
    b = dfpr.graph_load(n, src, dst, dfpr.default_config(precision=P))
    st = dfpr.static_pagerank(a, dfpr.default_params(mode=dfpr.JACOBI, tol=tol))
    assert st.status == dfpr.OK
    R0 = dfpr.get_ranks(a) * 1.25
    batch = workloads.uniform_batch(n, 40, 8, src, dst)
    for g in (a, b):
        dfpr.set_ranks(g, R0)
        dfpr.apply_batch(g, *batch)
    st_a = dfpr.df_pagerank(a, dfpr.default_params(mode=dfpr.JACOBI, normalize=1, tol=tol))
    st_b = dfpr.df_pagerank(b, dfpr.default_params(mode=dfpr.JACOBI, tol=tol))
    assert st_a.status == dfpr.OK and st_b.status == dfpr.OK
    assert st_a.passes == st_b.passes
    assert np.isnan(st_b.rank_sum)
    Ra, Rb = dfpr.get_ranks(a), dfpr.get_ranks(b)
    assert Rb.sum() > 1.01                     # the plain update kept most of the scale
    want = Rb / Rb.sum()
    if prec == "FP64":
        assert abs(st_a.rank_sum - 1.0) <= 1e-14
        assert abs(Ra.sum() - 1.0) <= 1e-14
        assert float(np.max(np.abs(Ra / want - 1.0))) <= 1e-14
    else:
        assert abs(st_a.rank_sum - 1.0) <= 1e-6
        assert float(np.max(np.abs(Ra / want - 1.0))) <= 1e-6
    for g in (a, b):
        g.free()
