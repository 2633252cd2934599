"""Pins for the CPU oracle: each check fixes the oracle against something other
than itself — closed forms of Eq. 1 on special graphs, a dense linear solve,
brute force on adjacency matrices, invariants, and the worked example of
Sec. 4.1.2. CPU only."""
import os

import numpy as np
import pytest

import oracle
import workloads

ALPHA = oracle.ALPHA
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Independent helpers (no oracle code)
# --------------------------------------------------------------------------

def adjacency(n, src, dst, self_loops=True):
    A = np.zeros((n, n), dtype=bool)
    A[np.asarray(src), np.asarray(dst)] = True
    if self_loops:
        A[np.arange(n), np.arange(n)] = True
    return A


def dense_pagerank(A, alpha=ALPHA, teleport=False):
    """Solves (I - alpha P^T) r = (1 - alpha)/n 1 with numpy's LU solver, where
    P[u, v] = 1/outdeg(u) for u -> v. With teleport=True the rank of dead ends
    is spread uniformly: r = alpha P^T r + alpha (d . r)/n 1 + (1 - alpha)/n 1."""
    n = A.shape[0]
    deg = A.sum(axis=1).astype(np.float64)
    P = np.zeros((n, n))
    nz = deg > 0
    P[nz] = A[nz] / deg[nz, None]
    M = alpha * P.T
    if teleport:
        M = M + alpha / n * np.outer(np.ones(n), (~nz).astype(np.float64))
    return np.linalg.solve(np.eye(n) - M, np.full(n, (1.0 - alpha) / n))


def edges_of(A):
    s, d = np.nonzero(A)
    return s.astype(np.int32), d.astype(np.int32)


def random_graph(n, p, rng):
    A = rng.random((n, n)) < p
    return edges_of(A)


# --------------------------------------------------------------------------
# Closed forms of Eq. 1
# --------------------------------------------------------------------------

@pytest.mark.parametrize("self_loops", [False, True])
@pytest.mark.parametrize("n", [3, 17, 64])
def test_directed_cycle_is_uniform(n, self_loops):
    src = np.arange(n, dtype=np.int32)
    dst = ((src + 1) % n).astype(np.int32)
    R, st = oracle.Graph.build(n, src, dst, self_loops).reference()
    assert np.max(np.abs(R - 1.0 / n)) < 1e-15
    assert st.converged


@pytest.mark.parametrize("n", [2, 9, 40])
def test_complete_digraph_is_uniform(n):
    u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = u != v
    R, _ = oracle.Graph.build(n, u[keep], v[keep], True).reference()
    assert np.max(np.abs(R - 1.0 / n)) < 1e-15


@pytest.mark.parametrize("n", [2, 5, 33, 200])
def test_directed_star_with_self_loops(n):
    # leaves 1..n-1 -> centre 0, self-loops everywhere
    src = np.arange(1, n, dtype=np.int32)
    dst = np.zeros(n - 1, np.int32)
    R, _ = oracle.Graph.build(n, src, dst, True).reference()
    a = ALPHA
    leaf = 2 * (1 - a) / (n * (2 - a))
    centre = (a * n + 2 - 2 * a) / (n * (2 - a))
    # rounding: n terms summed into the centre, amplified by 1/(1 - alpha)
    tol = n * np.finfo(float).eps / (1 - a)
    assert abs(R[0] - centre) < tol * centre
    assert np.max(np.abs(R[1:] - leaf)) < 1e-15
    assert abs(R.sum() - 1.0) < tol


@pytest.mark.parametrize("n", [3, 11, 101])
def test_bidirectional_star(n):
    leaves = np.arange(1, n, dtype=np.int32)
    src = np.concatenate([leaves, np.zeros(n - 1, np.int32)])
    dst = np.concatenate([np.zeros(n - 1, np.int32), leaves])
    a = ALPHA
    R0, _ = oracle.Graph.build(n, src, dst, False).reference()
    centre = (1 + a * (n - 1)) / (n * (1 + a))
    tol = n * np.finfo(float).eps / (1 - a)
    assert abs(R0[0] - centre) < tol
    assert np.max(np.abs(R0[1:] - (1 - centre) / (n - 1))) < tol
    R1, _ = oracle.Graph.build(n, src, dst, True).reference()
    leaf = 1.0 / (n + a * n / 2 - a)
    assert np.max(np.abs(R1[1:] - leaf)) < tol
    assert abs(R1[0] - (1 - (n - 1) * leaf)) < tol


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_static_bb_iterates_follow_jacobi_closed_form(k):
    # Directed star with self-loops: a leaf's only in-edge is its own loop
    # (out-degree 2), so the Jacobi iterate from 1/n is exactly
    # l_k = l* + (1/n - l*) (alpha/2)^k, and the centre follows
    # c_{k+1} = (1-a)/n + a c_k + a (n-1) l_k / 2.
    n = 7
    src = np.arange(1, n, dtype=np.int32)
    dst = np.zeros(n - 1, np.int32)
    g = oracle.Graph.build(n, src, dst, True)
    R, st = g.static_bb(max_iter=k, tol=0.0)
    a = ALPHA
    ls = 2 * (1 - a) / (n * (2 - a))
    leaf = [ls + (1.0 / n - ls) * (a / 2) ** j for j in range(k + 1)]
    c = 1.0 / n
    for j in range(k):
        c = (1 - a) / n + a * c + a * (n - 1) * leaf[j] / 2
    assert st.iterations == k
    assert np.max(np.abs(R[1:] - leaf[k])) < 1e-16
    assert abs(R[0] - c) < 1e-15


def test_single_vertex():
    R, _ = oracle.Graph.build(1, [], [], True).reference()
    assert abs(R[0] - 1.0) < 1e-15


# --------------------------------------------------------------------------
# Dense linear solve
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_reference_matches_dense_solve(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 65))
    src, dst = random_graph(n, rng.uniform(0.02, 0.3), rng)
    g = oracle.Graph.build(n, src, dst, True)
    R, st = g.reference()
    exact = dense_pagerank(adjacency(n, src, dst))
    assert np.max(np.abs(R - exact)) < 1e-13
    assert abs(R.sum() - 1.0) < 1e-12
    # Static_BB at tau = 1e-10 lands within the usual 1/(1 - alpha) bound
    R10, st10 = g.static_bb()
    assert st10.converged and st10.last_delta <= 1e-10
    assert np.max(np.abs(R10 - exact)) < 1e-10 / (1 - ALPHA)


@pytest.mark.parametrize("alpha", [0.5, 0.95])
@pytest.mark.parametrize("seed", range(3))
def test_other_damping_matches_dense_solve(seed, alpha):
    """The oracle's Static_BB and DF_BB at damping factors other than 0.85,
    which the GPU parity tests compare against."""
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 65))
    src, dst = random_graph(n, rng.uniform(0.02, 0.3), rng)
    g = oracle.Graph.build(n, src, dst, True)
    exact = dense_pagerank(adjacency(n, src, dst), alpha=alpha)
    R, _ = g.static_bb(alpha=alpha, tol=oracle.REF_TOL, max_iter=oracle.MAX_ITER)
    assert np.max(np.abs(R - exact)) < 1e-13
    # DF_BB after a batch of two insertions lands within the 1/(1 - alpha) bound
    A = adjacency(n, src, dst)
    ins = [(int(u), int(v)) for u, v in zip(*np.nonzero(~A))][:2]
    e = np.zeros(0, np.int32)
    batch = (e, e, np.array([u for u, _ in ins], np.int32), np.array([v for _, v in ins], np.int32))
    g1, _ = g.apply(*batch)
    R1, st = g1.df_bb(R, alpha=alpha)
    A1 = A.copy()
    for u, v in ins:
        A1[u, v] = True
    exact1 = dense_pagerank(A1, alpha=alpha)
    assert np.max(np.abs(R1 - exact1)) < oracle.TOL / (1 - alpha)


@pytest.mark.parametrize("seed", range(4))
def test_teleport_reading_matches_dense_solve(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 50))
    src, dst = random_graph(n, 0.08, rng)
    A = adjacency(n, src, dst, self_loops=False)
    A[0, :] = False  # at least one dead end
    s, d = edges_of(A)
    R, _ = oracle.Graph.build(n, s, d, False).reference(dead_end=1)
    exact = dense_pagerank(A, teleport=True)
    assert np.max(np.abs(R - exact)) < 1e-13
    assert abs(R.sum() - 1.0) < 1e-12


def teleport_case(seed, change_dead_ends):
    """A graph without self-loops and with dead ends, and a batch. With
    change_dead_ends the batch deletes every out-edge of a vertex (a new dead
    end) and inserts an edge out of an old dead end; otherwise it only adds
    edges between vertices that already have out-edges."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(20, 60))
    src, dst = random_graph(n, 0.08, rng)
    A = adjacency(n, src, dst, self_loops=False)
    A[0, :] = False                       # vertex 0 is a dead end
    A[1, :] = False
    A[1, 2] = True                        # vertex 1 has one out-edge
    A[np.arange(n), np.arange(n)] = False
    s, d = edges_of(A)
    live = [u for u in range(2, n) if A[u].any()]
    ins = []
    while len(ins) < 3:
        u, v = int(rng.choice(live)), int(rng.integers(0, n))
        if u != v and not A[u, v]:
            ins.append((u, v))
    dels = []
    if change_dead_ends:
        dels = [(1, 2)]                   # vertex 1 becomes a dead end
        ins.append((0, 3))                # vertex 0 is a dead end no more
    B = A.copy()
    for u, v in dels:
        B[u, v] = False
    for u, v in ins:
        B[u, v] = True
    arr = lambda pairs, k: np.array([p[k] for p in pairs], np.int32)  # noqa: E731
    batch = (arr(dels, 0), arr(dels, 1), arr(ins, 0), arr(ins, 1))
    return n, s, d, A, B, batch


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("change_dead_ends", [False, True])
def test_teleport_df_bb_matches_dense_solve(seed, change_dead_ends):
    n, s, d, A, B, batch = teleport_case(seed, change_dead_ends)
    g0 = oracle.Graph.build(n, s, d, False)
    R0, _ = g0.reference(dead_end=1)
    assert np.max(np.abs(R0 - dense_pagerank(A, teleport=True))) < 1e-13
    g1, _ = g0.apply(*batch)
    D_before = g0.dangling_mass(R0)
    assert abs(D_before - R0[~A.any(axis=1)].sum()) < 1e-15
    R1, st = g1.df_bb_teleport(R0, D_before)
    assert st.converged
    exact = dense_pagerank(B, teleport=True)
    assert np.max(np.abs(R1 - exact)) < 1e-9
    if change_dead_ends:
        # rank moved into and out of dead ends by far more than n * tol_f / alpha:
        # the shared term changed for every vertex, so every vertex is recomputed
        assert st.affected == n


def test_teleport_df_bb_without_change_is_identity():
    n, s, d, A, _, _ = teleport_case(0, False)
    g0 = oracle.Graph.build(n, s, d, False)
    R0, _ = g0.reference(dead_end=1)
    empty = np.zeros(0, np.int32)
    g1, _ = g0.apply(empty, empty, empty, empty)
    R1, st = g1.df_bb_teleport(R0, g0.dangling_mass(R0))
    assert st.affected == 0 and np.array_equal(R1, R0)


@pytest.mark.parametrize("seed", range(4))
def test_lock_free_static_matches_dense_solve(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 60))
    src, dst = random_graph(n, 0.1, rng)
    g = oracle.Graph.build(n, src, dst, True)
    R, st = g.static_lf(tol=1e-14)
    assert st.converged
    assert np.max(np.abs(R - dense_pagerank(adjacency(n, src, dst)))) < 1e-12


# --------------------------------------------------------------------------
# Graph update: brute force on adjacency matrices
# --------------------------------------------------------------------------

def brute_apply(A, ds, dd, is_, id_, self_loops):
    B = A.copy()
    for u, v in zip(ds, dd):
        if self_loops and u == v:
            continue
        B[u, v] = False
    for u, v in zip(is_, id_):
        B[u, v] = True
    real_del = A & ~B
    real_ins = B & ~A
    return B, real_del, real_ins


def check_csr_csc(g, B):
    n = B.shape[0]
    off, idx = g.csr()
    coff, cidx = g.csc()
    assert off[0] == 0 and off[-1] == B.sum() == g.m
    assert coff[-1] == g.m
    for u in range(n):
        row = idx[off[u]:off[u + 1]]
        assert np.array_equal(row, np.nonzero(B[u])[0]), u
        col = cidx[coff[u]:coff[u + 1]]
        assert np.array_equal(col, np.nonzero(B[:, u])[0]), u
    assert np.all(np.diff(off) >= 0) and np.all(np.diff(coff) >= 0)


@pytest.mark.parametrize("self_loops", [True, False])
@pytest.mark.parametrize("seed", range(8))
def test_graph_update_bruteforce(seed, self_loops):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 40))
    src, dst = random_graph(n, rng.uniform(0.0, 0.4), rng)
    # raw edges with duplicates
    if len(src):
        k = rng.integers(0, len(src), size=len(src) // 2)
        src = np.concatenate([src, src[k]])
        dst = np.concatenate([dst, dst[k]])
    A = adjacency(n, src, dst, self_loops)
    g = oracle.Graph.build(n, src, dst, self_loops)
    check_csr_csc(g, A)
    # batch with duplicates, no-ops, self-loop deletions, delete+reinsert pairs
    b = int(rng.integers(0, 3 * n + 1))
    ds = rng.integers(0, n, b).astype(np.int32)
    dd = rng.integers(0, n, b).astype(np.int32)
    is_ = rng.integers(0, n, b).astype(np.int32)
    id_ = rng.integers(0, n, b).astype(np.int32)
    if b:
        is_[: b // 4] = ds[: b // 4]
        id_[: b // 4] = dd[: b // 4]
        ds = np.concatenate([ds, ds[:3]])
        dd = np.concatenate([dd, dd[:3]])
        ds[-1] = dd[-1]
    B, rd, ri = brute_apply(A, ds, dd, is_, id_, self_loops)
    g1, nreal = g.apply(ds, dd, is_, id_)
    check_csr_csc(g1, B)
    assert nreal == (int(rd.sum()), int(ri.sum()))
    lds, ldd, lis, lid = g1.last_batch()
    assert np.array_equal(np.stack(np.nonzero(rd)), np.stack([lds, ldd]))
    assert np.array_equal(np.stack(np.nonzero(ri)), np.stack([lis, lid]))


def test_graph_update_rejects_bad_ids():
    g = oracle.Graph.build(4, [0, 1], [1, 2])
    with pytest.raises(RuntimeError):
        g.apply([0], [4], [], [])
    with pytest.raises(RuntimeError):
        oracle.Graph.build(4, [0, -1], [1, 2])


def test_sample_rows_match_full_model():
    n, src, dst = workloads.rmat_graph(10, 8, 5)
    batch = workloads.uniform_batch(n, 300, 6, src, dst)
    g1, _ = oracle.Graph.build(n, src, dst).apply(*batch)
    off, idx = g1.csr()
    coff, cidx = g1.csc()
    which = np.array([0, 5, 17, 1023, 400, 3], np.int32)
    rows = oracle.sample_rows(n, src, dst, which, "out", batch=batch)
    cols = oracle.sample_rows(n, src, dst, which, "in", batch=batch)
    for w, r, c in zip(which, rows, cols):
        assert np.array_equal(r, idx[off[w]:off[w + 1]])
        assert np.array_equal(c, cidx[coff[w]:coff[w + 1]])


# --------------------------------------------------------------------------
# Dynamic Frontier
# --------------------------------------------------------------------------

def brute_initial_affected(A, B):
    """Sec. 4.1: out-neighbours in G^{t-1} or G^t of every source of a change."""
    changed = A ^ B
    sources = np.nonzero(changed.any(axis=1))[0]
    va = np.zeros(A.shape[0], bool)
    for u in sources:
        va |= A[u] | B[u]
    return va


@pytest.mark.parametrize("self_loops", [True, False])
@pytest.mark.parametrize("seed", range(6))
def test_initial_affected_bruteforce(seed, self_loops):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(2, 50))
    src, dst = random_graph(n, 0.1, rng)
    A = adjacency(n, src, dst, self_loops)
    b = int(rng.integers(0, n))
    ds, dd = edges_of(A)
    pick = rng.integers(0, max(1, len(ds)), b) if len(ds) else np.zeros(0, int)
    ds, dd = ds[pick], dd[pick]
    is_ = rng.integers(0, n, b).astype(np.int32)
    id_ = rng.integers(0, n, b).astype(np.int32)
    B, _, _ = brute_apply(A, ds, dd, is_, id_, self_loops)
    g1, _ = oracle.Graph.build(n, src, dst, self_loops).apply(ds, dd, is_, id_)
    assert np.array_equal(g1.initial_affected().astype(bool), brute_initial_affected(A, B))


def load_worked_example():
    n, edges, batch, expect = 0, [], {"del": [], "ins": []}, {}
    with open(os.path.join(GOLDEN, "worked_example_sec4_1.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "e":
                edges.append((int(t[1]), int(t[2])))
            elif t[0] in ("del", "ins"):
                batch[t[0]].append((int(t[1]), int(t[2])))
            else:
                expect[t[0]] = sorted(int(x) for x in t[1:])
    return n, np.array(edges, np.int32), batch, expect


def test_worked_example_frontier():
    n, e, batch, expect = load_worked_example()
    g0 = oracle.Graph.build(n, e[:, 0], e[:, 1], self_loops=False)
    R0, _ = g0.reference()
    d = np.array(batch["del"], np.int32)
    i = np.array(batch["ins"], np.int32)
    g1, nreal = g0.apply(d[:, 0], d[:, 1], i[:, 0], i[:, 1])
    assert nreal == (1, 1)
    assert sorted(np.nonzero(g1.initial_affected())[0]) == expect["initial"]
    _, st, trace = g1.df_bb(R0, trace=2)
    assert sorted(np.nonzero(trace[0])[0]) == expect["initial"]
    assert sorted(np.nonzero(trace[1])[0]) == expect["after_first_iteration"]
    # sources of the change are not affected initially (no self-loops)
    assert trace[0][7] == 0 and trace[0][10] == 0


def rmat_case(scale=11, b=400, seed=7):
    n, src, dst = workloads.rmat_graph(scale, 16, seed)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.static_bb()
    batch = workloads.uniform_batch(n, b, seed + 1, src, dst)
    g1, _ = g0.apply(*batch)
    return n, g0, g1, R0, batch


@pytest.mark.parametrize("algo", ["df_bb", "df_lf"])
def test_df_matches_dense_solve(algo):
    n, g0, g1, R0, _ = rmat_case()
    off, idx = g1.csr()
    A = np.zeros((n, n), bool)
    A[np.repeat(np.arange(n), np.diff(off)), idx] = True
    exact = dense_pagerank(A)
    R, st = getattr(g1, algo)(R0)
    assert st.converged
    assert np.max(np.abs(R - exact)) < 1e-9        # paper's error bound (Sec. 5.2.2)
    assert 0 < st.affected < n


def test_df_empty_batch_is_identity():
    n, src, dst = workloads.rmat_graph(9, 8, 3)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.static_bb()
    e = np.zeros(0, np.int32)
    g1, nreal = g0.apply(e, e, e, e)
    assert nreal == (0, 0)
    for algo in ("df_bb", "df_lf"):
        R, st = getattr(g1, algo)(R0)
        assert st.processed == 0 and st.affected == 0
        assert np.array_equal(R, R0)


def test_df_bb_full_batch_equals_nd_bb():
    # one insertion out of every vertex: every vertex is affected from the start
    n, src, dst = workloads.rmat_graph(8, 8, 4)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.static_bb()
    u = np.arange(n, dtype=np.int32)
    v = ((u * 7 + 3) % n).astype(np.int32)
    g1, nreal = g0.apply([], [], u, v)
    assert np.all(g1.initial_affected() == 1)
    R_df, st_df = g1.df_bb(R0)
    R_nd, st_nd = g1.static_bb(R0)
    assert np.array_equal(R_df, R_nd)
    assert st_df.iterations == st_nd.iterations


def test_df_stability_round_trip():
    # Sec. 5.2.3: delete a batch, update, reinsert it, update; compare with original
    n, src, dst = workloads.rmat_graph(11, 16, 9)
    g0 = oracle.Graph.build(n, src, dst)
    R0, _ = g0.static_bb()
    ds, dd, _, _ = workloads.uniform_batch(n, 500, 10, src, dst, ins_frac=0.0)
    e = np.zeros(0, np.int32)
    for algo in ("df_bb", "df_lf"):
        g1, nr1 = g0.apply(ds, dd, e, e)
        R1, _ = getattr(g1, algo)(R0)
        g2, nr2 = g1.apply(e, e, ds, dd)
        assert nr1[0] == nr2[1] > 0
        R2, _ = getattr(g2, algo)(R1)
        assert np.array_equal(g2.csr()[1], g0.csr()[1])
        assert np.max(np.abs(R2 - R0)) < 1e-9


def test_df_respects_max_iterations():
    n, g0, g1, R0, _ = rmat_case(scale=9, b=100)
    R, st = g1.df_lf(R0, max_iter=2)
    assert st.iterations == 2 and not st.converged
    R, st = g1.df_bb(R0, max_iter=3)
    assert st.iterations == 3 and not st.converged


# --------------------------------------------------------------------------
# DF_LF's not-converged flags (Alg. 2, Sec. 4.3), derived by hand
# --------------------------------------------------------------------------

def test_df_lf_flags_keep_a_changed_source_for_one_more_pass():
    # G^0: 1 -> 0 (no self-loops), n = 3; the batch inserts 2 -> 0, so the
    # initial affected set is out(2) = {0}, flagged not converged (R_C = 1).
    # Pass 1 recomputes 0: its rank moves by alpha*b > tau (b = (1-alpha)/n),
    # so R_C[0] stays 1; 0 has no out-edges, so nothing else is marked.
    # Pass 2 recomputes 0 from unchanged inputs: the change is exactly 0, so
    # R_C[0] is cleared and the update stops. 2 passes, 2 recomputations of a
    # vertex with 2 in-edges; ranks follow Eq. 1 in closed form.
    n = 3
    b = (1.0 - ALPHA) / n
    g0 = oracle.Graph.build(n, [1], [0], self_loops=False)
    R0 = np.array([b * (1 + ALPHA), b, b])
    g1, nreal = g0.apply([], [], [2], [0])
    assert nreal == (0, 1)
    R, st = g1.df_lf(R0)
    assert st.converged
    assert st.iterations == 2
    assert st.processed == 2 and st.edges == 4
    assert st.affected == 1
    assert np.max(np.abs(R - np.array([b * (1 + 2 * ALPHA), b, b]))) < 1e-16


def test_df_lf_flags_follow_a_descending_chain():
    # G^0: 3 -> 2 -> 1 -> 0 (no self-loops), n = 5; the batch inserts 4 -> 3.
    # Ascending order visits a vertex before its in-neighbour on this chain, so
    # the change reaches one vertex further per pass:
    #   pass 1: {3} moves (alpha*b); marks 2 (VA = R_C = 1)
    #   pass 2: {2, 3}: 2 moves (alpha^2 b), marks 1; 3 does not move, clears
    #   pass 3: {1, 2, 3}: 1 moves, marks 0; 2 clears
    #   pass 4: {0, 1, 2, 3}: 0 moves (no out-edges); 1 clears
    #   pass 5: nothing moves; 0 clears; all flags clear -> stop.
    # 5 passes, 1+2+3+4+4 = 14 recomputations of in-degree-1 vertices, and
    # the exact ranks b * (1 + alpha + ... + alpha^k) along the chain.
    n = 5
    b = (1.0 - ALPHA) / n
    g0 = oracle.Graph.build(n, [3, 2, 1], [2, 1, 0], self_loops=False)
    geo = [sum(ALPHA ** j for j in range(k + 1)) for k in range(5)]
    R0 = b * np.array([geo[3], geo[2], geo[1], geo[0], geo[0]])
    g1, _ = g0.apply([], [], [4], [3])
    R, st = g1.df_lf(R0)
    assert st.converged
    assert st.iterations == 5
    assert st.processed == 14 and st.edges == 14
    assert st.affected == 4
    exact = b * np.array([geo[4], geo[3], geo[2], geo[1], geo[0]])
    assert np.max(np.abs(R - exact)) < 1e-16


def test_df_lf_tight_tolerance_matches_dense_solve():
    # With tau = 1e-14 the fixed point is reached to within a few 1e-14 per
    # vertex (error <= tau * (1 + alpha) / (1 - alpha) for a converged state),
    # so a pass that stops while a vertex still moves shows up here.
    n, g0, g1, R0, _ = rmat_case(scale=9, b=200, seed=21)
    off, idx = g1.csr()
    A = np.zeros((n, n), bool)
    A[np.repeat(np.arange(n), np.diff(off)), idx] = True
    exact = dense_pagerank(A)
    R_ref0, _ = g0.reference()          # R^{t-1} at FP64 rounding, not at tau
    R, st = g1.df_lf(R_ref0, tol=1e-14)
    assert st.converged
    assert np.max(np.abs(R - exact)) < 1e-12


# --------------------------------------------------------------------------
# Invariance under relabelling
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2])
def test_relabelling_permutes_ranks_and_work(seed):
    """Eq. 1 does not depend on vertex names: relabelling the graph, the batch
    and the starting ranks by a permutation permutes every rank, and leaves
    the DF iteration count and affected-set size unchanged. A mistake that
    ties a quantity to a vertex's position rather than to the vertex (an
    offset or degree read at the wrong index) breaks this."""
    rng = np.random.default_rng(seed)
    n, src, dst = workloads.rmat_graph(8, 8, 10 + seed)
    batch = workloads.uniform_batch(n, 40, 20 + seed, src, dst)
    perm = rng.permutation(n).astype(np.int32)
    g0 = oracle.Graph.build(n, src, dst)
    h0 = oracle.Graph.build(n, perm[src], perm[dst])
    R, _ = g0.reference()
    Rh, _ = h0.reference()
    assert np.max(np.abs(Rh[perm] - R)) <= 1e-15
    S, st = g0.static_bb()
    Sh, sth = h0.static_bb()
    assert st.iterations == sth.iterations
    assert np.max(np.abs(Sh[perm] - S)) <= 1e-15
    g1, nreal = g0.apply(*batch)
    h1, nreal_h = h0.apply(*[perm[np.asarray(x, np.int64)] for x in batch])
    assert nreal == nreal_h
    R0h = np.empty(n)
    R0h[perm] = R
    for algo in ("df_bb", "df_lf"):
        D, sd = getattr(g1, algo)(R)
        Dh, sdh = getattr(h1, algo)(R0h)
        assert sd.affected == sdh.affected
        if algo == "df_bb":  # deterministic Jacobi iterations
            assert sd.iterations == sdh.iterations
            assert np.max(np.abs(Dh[perm] - D)) <= 1e-15
        else:  # Alg. 2 visits vertices in id order: a different order, the same fixed point
            assert np.max(np.abs(Dh[perm] - D)) <= 1e-9
