"""Sets of graphs in one launch (dfpr_graph_load_parts): every graph of the
set must give what it gives alone, and what the oracle gives for it."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9


def make_set(specs, batch_frac=0.01, seed=500):
    """specs: list of (n, avg_degree). Returns per-graph data and the set's global arrays."""
    graphs = []
    off = [0]
    for i, (n, deg) in enumerate(specs):
        n, src, dst = workloads.rmat_graph_n(n, deg, seed + i)
        b = max(1, int(batch_frac * len(src)))
        batch = workloads.uniform_batch(n, b, seed + 100 + i, src, dst)
        graphs.append(dict(n=n, src=src, dst=dst, batch=batch))
        off.append(off[-1] + n)
    gsrc = np.concatenate([g["src"] + o for g, o in zip(graphs, off)]).astype(np.int32)
    gdst = np.concatenate([g["dst"] + o for g, o in zip(graphs, off)]).astype(np.int32)
    gbatch = [np.concatenate([g["batch"][k] + o for g, o in zip(graphs, off)]).astype(np.int32)
              for k in range(4)]
    return graphs, np.array(off, np.int32), gsrc, gdst, gbatch


SPECS = [(300, 6.0), (5000, 12.0), (20000, 4.0), (1000, 30.0), (70000, 9.0)]


@pytest.fixture(scope="module")
def gset():
    graphs, off, gsrc, gdst, gbatch = make_set(SPECS)
    for g in graphs:
        g0 = oracle.Graph.build(g["n"], g["src"], g["dst"])
        g1, nreal = g0.apply(*g["batch"])
        g["g0"], g["g1"], g["nreal"] = g0, g1, nreal
        g["ref0"], _ = g0.reference()
        g["ref1"], _ = g1.reference()
    return graphs, off, gsrc, gdst, gbatch


def test_set_structure_and_static(gpu_lib, gset):
    graphs, off, gsrc, gdst, _ = gset
    s = gpu_lib.graph_load_parts(off, gsrc, gdst)
    # CSR of the set = the graphs' CSRs with shifted ids
    goff, gidx = s.get_csr()
    for i, g in enumerate(graphs):
        o_off, o_idx = g["g0"].csr()
        a, b = off[i], off[i + 1]
        seg = gidx[goff[a]:goff[b]] - a
        assert np.array_equal(np.diff(goff[a:b + 1]), np.diff(o_off))
        assert np.array_equal(seg, o_idx)
    st = s.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI))
    assert st.status == gpu_lib.OK
    R = s.get_ranks()
    for i, g in enumerate(graphs):
        assert np.max(np.abs(R[off[i]:off[i + 1]] - g["ref0"])) <= LINF64, i


@pytest.mark.parametrize("mode", ["WORKLIST", "JACOBI"])
def test_set_df_matches_each_graph_alone(gpu_lib, gset, mode):
    graphs, off, gsrc, gdst, gbatch = gset
    s = gpu_lib.graph_load_parts(off, gsrc, gdst)
    s.set_ranks(np.concatenate([g["ref0"] for g in graphs]))
    got = s.apply_batch(*gbatch)
    assert got == tuple(map(sum, zip(*[g["nreal"] for g in graphs])))
    st = s.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
    assert st.status == gpu_lib.OK
    R = s.get_ranks()
    times = gpu_lib.get_part_times(s)
    assert times.shape == (len(graphs),) and np.all(times >= 0)
    for i, g in enumerate(graphs):
        Ri = R[off[i]:off[i + 1]]
        assert np.max(np.abs(Ri - g["ref1"])) <= LINF64, i
        # the same graph alone on the GPU
        alone = gpu_lib.graph_load(g["n"], g["src"], g["dst"])
        alone.set_ranks(g["ref0"])
        alone.apply_batch(*g["batch"])
        assert alone.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode))).status == gpu_lib.OK
        assert np.max(np.abs(alone.get_ranks() - Ri)) <= LINF64, i
        if mode == "WORKLIST":
            assert times[i] > 0


def test_set_graph_without_changes_does_no_work(gpu_lib, gset):
    graphs, off, gsrc, gdst, _ = gset
    s = gpu_lib.graph_load_parts(off, gsrc, gdst)
    s.set_ranks(np.concatenate([g["ref0"] for g in graphs]))
    g = graphs[1]
    b = [x + off[1] for x in g["batch"]]
    s.apply_batch(*[np.ascontiguousarray(x, np.int32) for x in b])
    assert s.df_pagerank().status == gpu_lib.OK
    times = gpu_lib.get_part_times(s)
    assert times[1] > 0
    assert all(times[i] == 0 for i in range(len(graphs)) if i != 1)
    R = s.get_ranks()
    for i in range(len(graphs)):
        if i != 1:
            assert np.array_equal(R[off[i]:off[i + 1]], graphs[i]["ref0"])


def test_set_rejects_edges_between_graphs(gpu_lib):
    off = np.array([0, 10, 20], np.int32)
    src = np.array([1, 12, 3], np.int32)
    dst = np.array([2, 5, 4], np.int32)  # 12 -> 5 crosses
    with pytest.raises(gpu_lib.DfprError) as e:
        gpu_lib.graph_load_parts(off, src, dst)
    assert e.value.status == gpu_lib.EINVAL


def test_set_df_finishes_despite_crashed_warps(gpu_lib, gset):
    """Helping in a many-graph launch: the claimed vertices of crash-stopped
    warps go back to the queue, and every graph still matches the oracle."""
    graphs, off, gsrc, gdst, gbatch = gset
    s = gpu_lib.graph_load_parts(off, gsrc, gdst)
    s.set_ranks(np.concatenate([g["ref0"] for g in graphs]))
    s.apply_batch(*gbatch)
    st = s.df_pagerank(gpu_lib.default_params(grid_ctas=8, fault_crash_warps=40, fault_seed=13))
    assert st.status == gpu_lib.OK
    R = s.get_ranks()
    for i, g in enumerate(graphs):
        assert np.max(np.abs(R[off[i]:off[i + 1]] - g["ref1"])) <= LINF64
