"""Size limits of the graph store and of the update kernels, on the GPU.

- More than 2^31 edges. Edge offsets and positions are 64-bit, and edge keys
  are counted with 32-bit prefix sums, so a graph may hold up to 2^32 - 2
  edges (self-loops included). An R-MAT graph of scale 26 with 40 draws per
  vertex (about 2.6G edges after de-duplication, plus 67M self-loops) is
  built, given one batch of 1e-4 |E|, updated, and checked as the full-size
  benchmark workload is: sampled CSR and CSC rows bit for bit, and Eq. 1 at
  sampled vertices, with rows and degrees from the oracle's row sampler.
- Degree limit. A warp adds the degrees of the 32 rows it holds in 32-bit
  integers, so updates need every in- and out-degree at most 2^25 - 1. Graphs
  with more vertices than that have their degrees tracked. An update on a
  graph with a larger degree returns EINVAL, and works again once a batch
  brings the degree back under the limit.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

ALPHA = 0.85
TOL = 1e-10
TOL_F = TOL / 1000
DRIFT = 10.0  # drift since the last expansion that forces one (worklist schedule)
DEG_LIMIT = (1 << 25) - 1


def star_ranks(n, leaves):
    """Closed forms for leaves 1..L -> centre 0, self-loops everywhere, the
    other vertices isolated: a leaf u solves r = (1-a)/n + a r / 2, an
    isolated vertex r = (1-a)/n + a r, and the centre
    r0 = (1-a)/n + a (r0 + L r_leaf / 2)."""
    leaf = 2.0 * (1.0 - ALPHA) / (n * (2.0 - ALPHA))
    iso = 1.0 / n
    centre = 1.0 / n + ALPHA * leaves / (n * (2.0 - ALPHA))
    return centre, leaf, iso


def check_star(R, n, leaves, tol_centre, tol_rest):
    centre, leaf, iso = star_ranks(n, leaves)
    assert abs(R[0] - centre) <= tol_centre, abs(R[0] - centre)
    assert np.max(np.abs(R[1:leaves + 1] - leaf)) <= tol_rest
    assert np.max(np.abs(R[leaves + 1:] - iso)) <= tol_rest


def centre_bound(leaves, tol_f):
    """How far the centre may end from its closed form. Every leaf has the
    same history, so their errors add up instead of cancelling. A leaf stops
    re-expanding once its change is at most tol_f, within
    tol_f (a/2) / (1 - a/2) of its fixed point. It may then drift by up to
    DRIFT tol_f more after the centre last read it. The centre carries
    a / (1 - a) times the sum over the leaves, through their contributions
    of r / 2, plus fixed-point rounding of L 2^-63 a / (1 - a)."""
    per_leaf = tol_f * (ALPHA / 2) / (1 - ALPHA / 2) + DRIFT * tol_f
    return ALPHA / (1 - ALPHA) * (leaves / 2 * per_leaf + leaves * 2.0 ** -63)


def test_degree_limit_checked_and_recovered(gpu_lib):
    n = (1 << 25) + 8
    leaves = DEG_LIMIT - 2          # centre in-degree = leaves + its self-loop
    src = np.arange(1, leaves + 1, dtype=np.int32)
    dst = np.zeros(leaves, np.int32)
    g = gpu_lib.graph_load(n, src, dst)
    # worklist schedule (the centre's 2^25-edge in-row is split into tokens).
    # A leaf depends only on itself and ends within tol_f (a/2) / (1 - a/2)
    # of its closed form; an isolated vertex starts at its rank, 1/n
    tol = 1e-13
    st = g.static_pagerank(gpu_lib.default_params(tol=tol))
    assert st.status == gpu_lib.OK
    bound = centre_bound(leaves, tol / 1000)
    check_star(g.get_ranks(), n, leaves, bound, 1e-15)

    # two isolated vertices join the star: the centre's in-degree becomes 2^25
    e = np.zeros(0, np.int32)
    ins_s = np.array([n - 1, n - 2], np.int32)
    ins_d = np.zeros(2, np.int32)
    assert g.apply_batch(e, e, ins_s, ins_d) == (0, 2)
    for call in (g.df_pagerank, g.nd_pagerank, g.static_pagerank):
        with pytest.raises(gpu_lib.DfprError) as err:
            call(gpu_lib.default_params())
        assert err.value.status == gpu_lib.EINVAL
        assert "2^25 - 1" in str(err.value)
    check_star(g.get_ranks(), n, leaves, bound, 1e-15)  # ranks untouched

    # undo the batch: the degree is back under the limit and updates run again
    assert g.apply_batch(ins_s, ins_d, e, e) == (2, 0)
    st = g.df_pagerank(gpu_lib.default_params())
    assert st.status == gpu_lib.OK
    # the update recomputes the centre and the two vertices, not the leaves:
    # the centre moves within 1e-13 a / (1 - a) of its fixed point given the
    # leaves as they are
    check_star(g.get_ranks(), n, leaves, bound + 1e-12, 1e-15)


def big_enough():
    import torch
    free_dev, _ = torch.cuda.mem_get_info()
    try:
        free_host = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        free_host = 0
    return free_dev >= 160 * 2**30 and free_host >= 96 * 2**30


def test_more_than_2_31_edges(gpu_lib):
    import torch
    if not big_enough():
        pytest.skip("needs 160 GiB of free device memory and 96 GiB of free host memory")
    n, src, dst = workloads.rmat_graph(26, 40, 5)
    b = 260000  # about 1e-4 |E|
    batch = workloads.uniform_batch(n, b, 6, src, dst)
    g = gpu_lib.graph_load(n, src, dst)
    m = g.info()["m"]
    assert (1 << 31) < m <= (1 << 32) - 2
    st0 = g.static_pagerank(gpu_lib.default_params(tol=TOL / 1000))
    assert st0.status == gpu_lib.OK
    g.apply_batch(*batch)
    st = g.df_pagerank(gpu_lib.default_params())
    assert st.status == gpu_lib.OK
    R = g.get_ranks()
    assert np.all(R > 0)

    rng = np.random.default_rng(55)
    hubs = np.argsort(np.bincount(dst, minlength=n))[-2:]
    sample = np.unique(np.concatenate([rng.integers(0, n, 400), hubs, batch[0][:20],
                                       batch[2][:20]])).astype(np.int32)
    m_now = g.info()["m"]
    dev = torch.device("cuda")
    for direction, export in (("out", g.get_csr), ("in", g.get_csc)):
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        idx = torch.empty(m_now, dtype=torch.int32, device=dev)
        export(off, idx)
        torch.cuda.synchronize()
        assert int(off[-1]) == m_now
        rows = oracle.sample_rows(n, src, dst, sample, direction, batch=batch)
        offs = off[torch.from_numpy(sample.astype(np.int64)).to(dev)].cpu().numpy()
        ends = off[torch.from_numpy(sample.astype(np.int64) + 1).to(dev)].cpu().numpy()
        for v, lo, hi, row in zip(sample, offs, ends, rows):
            assert np.array_equal(idx[int(lo):int(hi)].cpu().numpy(), row), (direction, int(v))
        del off, idx

    # Eq. 1 at random vertices and at targets of inserted edges (see the
    # full-size test for the bound)
    resid = np.unique(np.concatenate([rng.integers(0, n, 100), batch[3][:10]])).astype(np.int32)
    rin = oracle.sample_rows(n, src, dst, resid, "in", batch=batch)
    nbrs = np.unique(np.concatenate(rin)).astype(np.int32)
    nbr_deg = np.array([len(r) for r in oracle.sample_rows(n, src, dst, nbrs, "out", batch=batch,
                                                           cap=1 << 26)], np.float64)
    for v, row in zip(resid, rin):
        d = nbr_deg[np.searchsorted(nbrs, row)]
        r = (1.0 - ALPHA) / n + ALPHA * float(np.sum(R[row] / d))
        bound = ALPHA * 2.0 * DRIFT * TOL_F * float(np.sum(1.0 / d)) + TOL / 1000 + 1e-14
        assert abs(r - R[v]) <= bound, (int(v), abs(r - R[v]), bound)
