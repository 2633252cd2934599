"""DF updates with teleport dead ends (no self-loops; the rank of dead ends is
spread over all vertices) on the GPU's jacobi schedule, against the oracle's
DF_BB with the same reading and against the reference ranks."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9


def small_case(seed, change_dead_ends):
    """Same construction as the oracle pins: a graph with dead ends and a
    batch that does or does not move vertices into / out of the dead-end set."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(20, 60))
    A = rng.random((n, n)) < 0.08
    A[0, :] = False
    A[1, :] = False
    A[1, 2] = True
    A[np.arange(n), np.arange(n)] = False
    s, d = (x.astype(np.int32) for x in np.nonzero(A))
    live = [u for u in range(2, n) if A[u].any()]
    ins = []
    while len(ins) < 3:
        u, v = int(rng.choice(live)), int(rng.integers(0, n))
        if u != v and not A[u, v]:
            ins.append((u, v))
    dels = []
    if change_dead_ends:
        dels = [(1, 2)]
        ins.append((0, 3))
    arr = lambda pairs, k: np.array([p[k] for p in pairs], np.int32)  # noqa: E731
    return n, s, d, (arr(dels, 0), arr(dels, 1), arr(ins, 0), arr(ins, 1))


def run_both(gpu_lib, n, s, d, batch):
    g0 = oracle.Graph.build(n, s, d, False)
    R0, _ = g0.reference(dead_end=1)
    g1, _ = g0.apply(*batch)
    ref1, _ = g1.reference(dead_end=1)
    orc, orc_st = g1.df_bb_teleport(R0, g0.dangling_mass(R0))
    cfg = gpu_lib.default_config(dead_end=gpu_lib.TELEPORT)
    g = gpu_lib.graph_load(n, s, d, cfg)
    g.set_ranks(R0)
    g.apply_batch(*batch)
    st = g.df_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI))
    return g.get_ranks(), st, orc, orc_st, ref1


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("change_dead_ends", [False, True])
def test_small_graphs_match_oracle_and_reference(gpu_lib, seed, change_dead_ends):
    n, s, d, batch = small_case(seed, change_dead_ends)
    R, st, orc, orc_st, ref1 = run_both(gpu_lib, n, s, d, batch)
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(R - ref1)) <= LINF64
    assert np.max(np.abs(R - orc)) <= 1e-12
    assert st.passes == orc_st.iterations
    if change_dead_ends:
        assert st.affected == n == orc_st.affected


def rmat_no_loops(scale, seed):
    n, src, dst = workloads.rmat_graph(scale, 16, seed)
    keep = src != dst
    return n, src[keep], dst[keep]


def test_rmat_batch_that_moves_dead_end_mass(gpu_lib):
    """Random batch on R-MAT scale 14 without self-loops: insertions out of dead
    ends move far more than n * tol_f / alpha of rank, so every vertex is
    recomputed, on both sides."""
    n, src, dst = rmat_no_loops(14, 21)
    batch = workloads.uniform_batch(n, 1000, 22, src, dst)
    R, st, orc, orc_st, ref1 = run_both(gpu_lib, n, src, dst, batch)
    assert st.status == gpu_lib.OK
    assert st.affected == n == orc_st.affected
    assert np.max(np.abs(R - ref1)) <= LINF64
    assert np.max(np.abs(R - orc)) <= 1e-11


def test_rmat_batch_between_live_vertices(gpu_lib):
    """Insertions only between vertices that already have out-edges: no vertex
    enters or leaves the dead-end set, so the update starts from the usual
    frontier and still lands on the reference."""
    n, src, dst = rmat_no_loops(14, 23)
    outdeg = np.bincount(src, minlength=n)
    live = np.nonzero(outdeg > 0)[0].astype(np.int32)
    rng = np.random.default_rng(24)
    ins_s = rng.choice(live, 400).astype(np.int32)
    ins_d = rng.choice(live, 400).astype(np.int32)
    keep = ins_s != ins_d
    empty = np.zeros(0, np.int32)
    batch = (empty, empty, ins_s[keep], ins_d[keep])
    R, st, orc, orc_st, ref1 = run_both(gpu_lib, n, src, dst, batch)
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(R - ref1)) <= LINF64
    assert np.max(np.abs(R - orc)) <= 1e-11


def test_teleport_rejects_other_schedules(gpu_lib):
    n, s, d, batch = small_case(0, False)
    g = gpu_lib.graph_load(n, s, d, gpu_lib.default_config(dead_end=gpu_lib.TELEPORT))
    g.apply_batch(*batch)
    for mode in ("WORKLIST", "ROUND"):
        with pytest.raises(gpu_lib.DfprError) as e:
            g.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
        assert e.value.status == gpu_lib.EINVAL
