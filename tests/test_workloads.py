"""The seeded generators: deterministic, in range, and shaped as specified."""
import numpy as np

import workloads


def test_rmat_deterministic_and_in_range():
    n, s1, d1 = workloads.rmat_graph(12, 8, 42)
    _, s2, d2 = workloads.rmat_graph(12, 8, 42)
    _, s3, _ = workloads.rmat_graph(12, 8, 43)
    assert n == 4096 and len(s1) == 8 * 4096
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert not np.array_equal(s1, s3)
    assert s1.min() >= 0 and s1.max() < n and d1.min() >= 0 and d1.max() < n


def test_rmat_is_skewed():
    # a = 0.57 concentrates draws: the top out-degree is far above the mean
    n, s, d = workloads.rmat_graph(14, 16, 1)
    deg = np.bincount(s, minlength=n)
    assert deg.max() > 20 * deg.mean()


def test_rmat_non_power_of_two():
    n, s, d = workloads.rmat_graph_n(3000, 10.0, 5)
    assert n == 3000 and s.max() < n and d.max() < n
    assert 0.5 * 10 * n < len(s) < 2 * 10 * n


def test_grid_structure():
    L = 16
    n, s, d = workloads.grid_graph(L, 3, shortcut_frac=0.01)
    grid = 4 * L * (L - 1)
    assert n == L * L and len(s) == grid + round(0.01 * grid)
    r1, c1, r2, c2 = s[:grid] // L, s[:grid] % L, d[:grid] // L, d[:grid] % L
    assert np.all(np.abs(r1 - r2) + np.abs(c1 - c2) == 1)
    keys = set(zip(s[:grid].tolist(), d[:grid].tolist()))
    assert all((b, a) in keys for a, b in keys)          # bidirectional
    assert np.all(s[grid:] != d[grid:])


def test_uniform_batch():
    n, s, d = workloads.rmat_graph(10, 8, 1)
    ds, dd, is_, id_ = workloads.uniform_batch(n, 1000, 2, s, d)
    assert len(is_) == 800 and len(ds) == 200
    assert np.all(is_ != id_) and is_.max() < n
    pool = set(zip(s.tolist(), d.tolist()))
    assert all(p in pool for p in zip(ds.tolist(), dd.tolist()))
    assert np.all(ds != dd)
    again = workloads.uniform_batch(n, 1000, 2, s, d)
    assert all(np.array_equal(a, b) for a, b in zip((ds, dd, is_, id_), again))


def test_grid_local_batch():
    L = 64
    ds, dd, is_, id_ = workloads.grid_local_batch(L, 50, 9)
    w = int(np.ceil(4 * np.sqrt(50)))
    pts = np.concatenate([ds, dd, is_, id_])
    assert np.ptp(pts // L) < w and np.ptp(pts % L) < w
    assert np.all(np.abs(ds // L - dd // L) + np.abs(ds % L - dd % L) == 1)
    assert len(is_) == 40 and len(ds) == 10


def test_many_graph_specs():
    specs = workloads.many_graph_specs(256, 1000)
    n = np.array([x[0] for x in specs])
    deg = np.array([x[1] for x in specs])
    assert n.min() >= 1000 and n.max() <= 1_000_000
    assert deg.min() >= 4 and deg.max() <= 32
