"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs. Graph structure and the initial frontier are compared bit
for bit; ranks within the paper's error bound, L-inf <= 1e-9 in FP64 (Sec.
5.2.2) and <= 1e-6 relative per vertex in FP32."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9
REL32 = 1e-6


def rmat_case(scale, b, seed=1, edge_factor=16):
    n, src, dst = workloads.rmat_graph(scale, edge_factor, seed)
    batch = workloads.uniform_batch(n, b, seed + 1, src, dst)
    return n, src, dst, batch


@pytest.fixture(scope="module")
def c1():
    """R-MAT scale 14, 16 draws per vertex, one batch of 1,000 edges (800 ins / 200 del)."""
    n, src, dst, batch = rmat_case(14, 1000)
    g0 = oracle.Graph.build(n, src, dst)
    g1, nreal = g0.apply(*batch)
    R0, _ = g0.static_bb()          # converged to tau = 1e-10, as the paper's runs
    R0ref, _ = g0.reference()       # converged to rounding
    ref1, _ = g1.reference()
    return dict(n=n, src=src, dst=dst, batch=batch, g0=g0, g1=g1, nreal=nreal, R0=R0,
                R0ref=R0ref, ref1=ref1)


def check_graph(gpu_g, orc_g):
    off, idx = gpu_g.get_csr()
    ooff, oidx = orc_g.csr()
    assert np.array_equal(off, ooff), "CSR offsets differ"
    assert np.array_equal(idx, oidx), "CSR ids differ"
    coff, cidx = gpu_g.get_csc()
    ocoff, ocidx = orc_g.csc()
    assert np.array_equal(coff, ocoff), "CSC offsets differ"
    assert np.array_equal(cidx, ocidx), "CSC ids differ"


# --------------------------------------------------------------------------
# Graph store (bit-exact)
# --------------------------------------------------------------------------

def test_graph_load_bit_exact(gpu_lib, c1):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    check_graph(g, c1["g0"])
    assert g.info()["m"] == c1["g0"].m


@pytest.mark.parametrize("n,m", [(1, 0), (2, 0), (3, 5), (37, 0), (64, 4000), (2049, 9000)])
def test_graph_load_edge_cases(gpu_lib, n, m):
    rng = np.random.default_rng(n * 7 + m)
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    for loops in (True, False):
        cfg = gpu_lib.default_config(dead_end=gpu_lib.SELF_LOOPS if loops else gpu_lib.TELEPORT)
        g = gpu_lib.graph_load(n, src, dst, cfg)
        check_graph(g, oracle.Graph.build(n, src, dst, loops))


def test_graph_load_rejects_bad_ids(gpu_lib):
    with pytest.raises(gpu_lib.DfprError) as e:
        gpu_lib.graph_load(10, np.array([1, 10], np.int32), np.array([2, 3], np.int32))
    assert e.value.status == gpu_lib.EINVAL


def test_apply_batch_bit_exact_sequence(gpu_lib, c1):
    """Several batches in a row, including duplicates, no-ops, self-loop deletions
    and an edge both deleted and inserted."""
    n, src, dst = c1["n"], c1["src"], c1["dst"]
    g = gpu_lib.graph_load(n, src, dst)
    og = c1["g0"]
    for k in range(4):
        ds, dd, is_, id_ = workloads.uniform_batch(n, 300 + 500 * k, 50 + k, src, dst)
        ds = np.concatenate([ds, ds[:5], np.array([7, 9], np.int32)])
        dd = np.concatenate([dd, dd[:5], np.array([7, 1], np.int32)])
        is_ = np.concatenate([is_, ds[:3], is_[:4]])
        id_ = np.concatenate([id_, dd[:3], id_[:4]])
        got = g.apply_batch(ds, dd, is_, id_)
        og, want = og.apply(ds, dd, is_, id_)
        assert got == want
        check_graph(g, og)


@pytest.mark.parametrize("loops", [True, False])
def test_apply_batch_overflow_rebuild(gpu_lib, loops):
    """No slack at all: every growing row relocates, the spare area runs out and
    the direction is rebuilt; the result must still match bit for bit."""
    n, src, dst, _ = rmat_case(11, 0, seed=5, edge_factor=8)
    cfg = gpu_lib.default_config(row_slack=0.0, min_slack=0, tail_slack=0.0,
                                 dead_end=gpu_lib.SELF_LOOPS if loops else gpu_lib.TELEPORT)
    g = gpu_lib.graph_load(n, src, dst, cfg)
    og = oracle.Graph.build(n, src, dst, loops)
    for k in range(3):
        batch = workloads.uniform_batch(n, 4000, 70 + k, src, dst, ins_frac=0.9)
        got = g.apply_batch(*batch)
        og, want = og.apply(*batch)
        assert got == want
        check_graph(g, og)


def test_apply_batch_rejects_bad_ids_and_keeps_graph(gpu_lib, c1):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    bad = np.array([0, c1["n"]], np.int32)
    with pytest.raises(gpu_lib.DfprError) as e:
        g.apply_batch(bad, bad, bad[:0], bad[:0])
    assert e.value.status == gpu_lib.EINVAL
    check_graph(g, c1["g0"])


def test_apply_batch_device_arrays(gpu_lib, c1):
    import torch
    g = gpu_lib.graph_load(c1["n"], torch.from_numpy(c1["src"]).cuda(), torch.from_numpy(c1["dst"]).cuda())
    batch = [torch.from_numpy(x).cuda() for x in c1["batch"]]
    assert g.apply_batch(*batch) == c1["nreal"]
    check_graph(g, c1["g1"])


# --------------------------------------------------------------------------
# Initial marking (bit-exact)
# --------------------------------------------------------------------------

def test_initial_affected_bit_exact(gpu_lib, c1):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    g.apply_batch(*c1["batch"])
    flags, count = g.initial_affected()
    want = c1["g1"].initial_affected()
    assert np.array_equal(flags, want)
    assert count == int(want.sum())
    # marking alone leaves no trace: a second call gives the same flags
    flags2, _ = g.initial_affected()
    assert np.array_equal(flags2, want)


def test_initial_affected_worked_example(gpu_lib):
    from tests.test_oracle_pins import load_worked_example
    n, e, batch, expect = load_worked_example()
    cfg = gpu_lib.default_config(dead_end=gpu_lib.TELEPORT)  # the example has no self-loops
    g = gpu_lib.graph_load(n, e[:, 0].copy(), e[:, 1].copy(), cfg)
    d = np.array(batch["del"], np.int32)
    i = np.array(batch["ins"], np.int32)
    assert g.apply_batch(d[:, 0].copy(), d[:, 1].copy(), i[:, 0].copy(), i[:, 1].copy()) == (1, 1)
    flags, count = g.initial_affected()
    assert sorted(np.nonzero(flags)[0]) == expect["initial"] and count == 3


def test_pending_changes_accumulate(gpu_lib, c1):
    """Two batches before one update mark the union of their frontiers."""
    n, src, dst = c1["n"], c1["src"], c1["dst"]
    b1 = workloads.uniform_batch(n, 100, 91, src, dst)
    b2 = workloads.uniform_batch(n, 100, 92, src, dst)
    g = gpu_lib.graph_load(n, src, dst)
    g.apply_batch(*b1)
    g.apply_batch(*b2)
    flags, _ = g.initial_affected()
    o1, _ = c1["g0"].apply(*b1)
    o2, _ = o1.apply(*b2)
    want = o1.initial_affected() | o2.initial_affected()
    assert np.array_equal(flags, want)


# --------------------------------------------------------------------------
# Ranks
# --------------------------------------------------------------------------

MODES = ["WORKLIST", "ROUND", "JACOBI"]


@pytest.mark.parametrize("mode", MODES)
def test_static_matches_reference(gpu_lib, c1, mode):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    st = g.static_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
    assert st.status == gpu_lib.OK
    ref0, _ = c1["g0"].reference()
    assert np.max(np.abs(g.get_ranks() - ref0)) <= LINF64


@pytest.mark.parametrize("mode", MODES)
def test_df_matches_reference(gpu_lib, c1, mode):
    """R^{t-1} converged to rounding (the oracle's reference on G^{t-1}), then
    one DF update: the error is the DF schedule's own. (Starting from ranks
    converged only to tau = 1e-10 already spends ~5e-10 of the 1e-9 budget;
    that full path is covered by test_df_after_gpu_static.)"""
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    g.set_ranks(c1["R0ref"])
    assert g.apply_batch(*c1["batch"]) == c1["nreal"]
    st = g.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
    assert st.status == gpu_lib.OK, st.as_dict()
    R = g.get_ranks()
    err = np.max(np.abs(R - c1["ref1"]))
    assert err <= LINF64, err
    assert 0 < st.processed and 0 < st.affected <= c1["n"]


def test_df_jacobi_matches_oracle_df_bb(gpu_lib, c1):
    """Alg. 1 with marks effective from the next iteration is deterministic: same
    iteration count and affected set as the oracle's DF_BB, values to rounding."""
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    g.set_ranks(c1["R0"])
    g.apply_batch(*c1["batch"])
    st = g.df_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI))
    R_o, st_o = c1["g1"].df_bb(c1["R0"])
    assert st.passes == st_o.iterations
    assert st.affected == st_o.affected
    assert np.max(np.abs(g.get_ranks() - R_o)) <= 1e-13


@pytest.mark.parametrize("split", [256, 1024])
def test_df_jacobi_split_rows_match_oracle_df_bb(gpu_lib, c1, split):
    """Long in-rows summed in chunks by many warps (every in-row above `split`
    edges): the same iterations, affected set and values as the oracle's
    DF_BB; the integer fixed-point sums make the chunk order irrelevant."""
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    indeg = np.diff(g.get_csc()[0])
    assert (indeg > split).sum() >= 4  # the case has split rows
    g.set_ranks(c1["R0"])
    g.apply_batch(*c1["batch"])
    st = g.df_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI, gather_split=split))
    R_o, st_o = c1["g1"].df_bb(c1["R0"])
    assert st.passes == st_o.iterations
    assert st.affected == st_o.affected
    assert np.max(np.abs(g.get_ranks() - R_o)) <= 1e-13
    # static (every vertex, every iteration) with split rows
    st = g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI, gather_split=split))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - c1["ref1"])) <= LINF64


def test_df_after_gpu_static(gpu_lib, c1):
    """The whole path on the GPU: static ranks, batch, DF."""
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    assert g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI)).status == gpu_lib.OK
    g.apply_batch(*c1["batch"])
    st = g.df_pagerank()
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - c1["ref1"])) <= LINF64


def test_df_empty_batch(gpu_lib, c1):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    g.set_ranks(c1["R0"])
    st = g.df_pagerank()
    assert st.processed == 0 and st.status == gpu_lib.OK
    assert np.array_equal(g.get_ranks(), c1["R0"])
    e = np.zeros(0, np.int32)
    assert g.apply_batch(e, e, e, e) == (0, 0)
    st = g.df_pagerank()
    assert st.processed == 0
    # a batch of no-ops (an absent deletion, a self-loop deletion, present
    # insertions) changes nothing and leaves nothing to update
    off, idx = c1["g0"].csr()
    u = 3
    row = set(idx[off[u]:off[u + 1]].tolist())
    absent = next(w for w in range(c1["n"]) if w not in row)
    present = np.array(sorted(row)[:2], np.int32)
    got = g.apply_batch(np.array([u, u], np.int32), np.array([absent, u], np.int32),
                        np.full(len(present), u, np.int32), present)
    assert got == (0, 0)
    assert g.df_pagerank().processed == 0
    check_graph(g, c1["g0"])


def test_df_sequence_of_batches(gpu_lib, c1):
    n, src, dst = c1["n"], c1["src"], c1["dst"]
    g = gpu_lib.graph_load(n, src, dst)
    g.set_ranks(c1["R0"])
    og = c1["g0"]
    for k in range(3):
        batch = workloads.uniform_batch(n, 500, 200 + k, src, dst)
        g.apply_batch(*batch)
        og, _ = og.apply(*batch)
        assert g.df_pagerank().status == gpu_lib.OK
    ref, _ = og.reference()
    assert np.max(np.abs(g.get_ranks() - ref)) <= LINF64


def test_df_stability_round_trip(gpu_lib, c1):
    """Sec. 5.2.3: delete a batch, update, reinsert it, update."""
    n, src, dst = c1["n"], c1["src"], c1["dst"]
    ds, dd, _, _ = workloads.uniform_batch(n, 2000, 33, src, dst, ins_frac=0.0)
    e = np.zeros(0, np.int32)
    g = gpu_lib.graph_load(n, src, dst)
    g.set_ranks(c1["R0"])
    g.apply_batch(ds, dd, e, e)
    assert g.df_pagerank().status == gpu_lib.OK
    g.apply_batch(e, e, ds, dd)
    assert g.df_pagerank().status == gpu_lib.OK
    check_graph(g, c1["g0"])
    assert np.max(np.abs(g.get_ranks() - c1["R0"])) <= LINF64


def test_nd_matches_reference(gpu_lib, c1):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    g.set_ranks(c1["R0"])
    g.apply_batch(*c1["batch"])
    for mode in MODES:
        g.set_ranks(c1["R0"])
        st = g.nd_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
        assert st.status == gpu_lib.OK
        assert np.max(np.abs(g.get_ranks() - c1["ref1"])) <= LINF64


def test_fp32_relative_error(gpu_lib, c1):
    cfg = gpu_lib.default_config(precision=gpu_lib.FP32)
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"], cfg)
    p = gpu_lib.default_params(tol=1e-7)
    assert g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI, tol=1e-7)).status == gpu_lib.OK
    g.apply_batch(*c1["batch"])
    st = g.df_pagerank(p)
    assert st.status == gpu_lib.OK
    R = g.get_ranks()
    rel = np.abs(R - c1["ref1"]) / c1["ref1"]
    assert np.max(rel) <= REL32, np.max(rel)


def test_teleport_static_matches_reference(gpu_lib):
    rng = np.random.default_rng(4)
    n = 3000
    src = rng.integers(0, n, 9000).astype(np.int32)
    dst = rng.integers(0, n, 9000).astype(np.int32)
    g = gpu_lib.graph_load(n, src, dst, gpu_lib.default_config(dead_end=gpu_lib.TELEPORT))
    st = g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI))
    assert st.status == gpu_lib.OK
    ref, _ = oracle.Graph.build(n, src, dst, False).reference(dead_end=1)
    assert np.max(np.abs(g.get_ranks() - ref)) <= LINF64
    # the worklist and round schedules need self-loops (no global dead-end term)
    with pytest.raises(gpu_lib.DfprError):
        g.df_pagerank()
    with pytest.raises(gpu_lib.DfprError):
        g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.WORKLIST))


def test_timeout_returns_status_and_recovers(gpu_lib, c1):
    """A budget too small to finish: the kernel gives up on its own, reports
    ETIMEOUT, and the graph stays usable."""
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    g.set_ranks(c1["R0"])
    g.apply_batch(*c1["batch"])
    st = g.df_pagerank(gpu_lib.default_params(timeout_ms=1e-6))
    assert st.status in (gpu_lib.ETIMEOUT, gpu_lib.OK)
    st = g.nd_pagerank()
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - c1["ref1"])) <= LINF64


def test_iteration_cap_returns_notconv(gpu_lib, c1):
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"])
    st = g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI, max_iter=3))
    assert st.status == gpu_lib.ENOTCONV and st.passes == 3
    st = g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.ROUND, max_iter=2))
    assert st.status == gpu_lib.ENOTCONV


# --------------------------------------------------------------------------
# Medium size: several thousand tiles, oracle still in seconds
# --------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_df_rmat18(gpu_lib, precision):
    n, src, dst, batch = rmat_case(18, 4000, seed=11)
    g0 = oracle.Graph.build(n, src, dst)
    g1, nreal = g0.apply(*batch)
    ref1, _ = g1.reference()
    cfg = gpu_lib.default_config(precision=getattr(gpu_lib, precision))
    g = gpu_lib.graph_load(n, src, dst, cfg)
    tol = 1e-10 if precision == "FP64" else 1e-7
    assert g.static_pagerank(gpu_lib.default_params(mode=gpu_lib.JACOBI, tol=tol)).status == gpu_lib.OK
    assert g.apply_batch(*batch) == nreal
    check_graph(g, g1)
    st = g.df_pagerank(gpu_lib.default_params(tol=tol))
    assert st.status == gpu_lib.OK
    R = g.get_ranks()
    if precision == "FP64":
        assert np.max(np.abs(R - ref1)) <= LINF64
    else:
        assert np.max(np.abs(R - ref1) / ref1) <= REL32


def test_grid_local_batch(gpu_lib):
    L = 256
    n, src, dst = workloads.grid_graph(L, 4)
    batch = workloads.grid_local_batch(L, 300, 5)
    g0 = oracle.Graph.build(n, src, dst)
    g1, nreal = g0.apply(*batch)
    # R^{t-1} converged below the frontier tolerance: with ranks converged only
    # to tau, every recomputed vertex moves by more than tau_f = tau / 1000 and
    # the frontier spreads over the whole graph whatever the batch
    R0, _ = g0.reference()
    ref1, _ = g1.reference()
    g = gpu_lib.graph_load(n, src, dst)
    g.set_ranks(R0)
    assert g.apply_batch(*batch) == nreal
    check_graph(g, g1)
    st = g.df_pagerank()
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - ref1)) <= LINF64
    assert st.affected < n // 2  # a localised batch touches a small region


@pytest.mark.parametrize("reorder", [0, 1])
def test_caller_numbering_kept_with_and_without_reorder(gpu_lib, c1, reorder):
    """The internal degree ordering is invisible at the interface: graph exports,
    ranks and the initial frontier come back in the caller's ids either way."""
    cfg = gpu_lib.default_config(reorder=reorder)
    g = gpu_lib.graph_load(c1["n"], c1["src"], c1["dst"], cfg)
    check_graph(g, c1["g0"])
    g.set_ranks(c1["R0ref"])
    assert np.array_equal(g.get_ranks(), c1["R0ref"])
    assert g.apply_batch(*c1["batch"]) == c1["nreal"]
    check_graph(g, c1["g1"])
    flags, _ = g.initial_affected()
    assert np.array_equal(flags, c1["g1"].initial_affected())
    st = g.df_pagerank()
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - c1["ref1"])) <= LINF64


# --------------------------------------------------------------------------
# Batch sizes at the ends of the range
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", MODES)
def test_df_large_batch(gpu_lib, c1, mode):
    """A batch of 10 % of the edges (the top of the swept range): most
    vertices are affected; every schedule still lands on the reference."""
    n, src, dst = c1["n"], c1["src"], c1["dst"]
    batch = workloads.uniform_batch(n, 26000, 41, src, dst)
    g1, nreal = c1["g0"].apply(*batch)
    ref1, _ = g1.reference()
    g = gpu_lib.graph_load(n, src, dst)
    g.set_ranks(c1["R0ref"])
    assert g.apply_batch(*batch) == nreal
    check_graph(g, g1)
    st = g.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - ref1)) <= LINF64


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,edges,batch", [
    (1, [], ([], [], [], [])),                          # one vertex, only its self-loop
    (2, [(0, 1)], ([0], [1], [1], [0])),                 # the only edge turns around
    (5, [(0, 1), (1, 2), (2, 3), (3, 4)], ([1], [2], [4, 4], [0, 2])),
])
def test_df_tiny_graphs(gpu_lib, mode, n, edges, batch):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    b = tuple(np.array(x, np.int32) for x in batch)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.reference()
    g1, nreal = g0.apply(*b)
    ref1, _ = g1.reference()
    g = gpu_lib.graph_load(n, src, dst)
    g.set_ranks(R0)
    assert g.apply_batch(*b) == nreal
    check_graph(g, g1)
    st = g.df_pagerank(gpu_lib.default_params(mode=getattr(gpu_lib, mode)))
    assert st.status == gpu_lib.OK
    assert np.max(np.abs(g.get_ranks() - ref1)) <= LINF64
