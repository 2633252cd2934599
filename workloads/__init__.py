"""Seeded synthetic inputs shared by the CPU oracle's tests and the GPU path.

This module draws random graphs and edge-update batches; it holds none of the
PageRank arithmetic and builds no graph structure. The generators live in
``gen.c`` (SplitMix64, counter-based, so the output does not depend on the
thread count) and are compiled on first use with the host C compiler.

Workload recipes (stand-ins for the paper's datasets, Sec. 5.1.3, Table 2,
and its batch generation, Sec. 5.1.4):

* ``rmat_graph(scale, edge_factor, seed)``: R-MAT with a, b, c, d =
  0.57, 0.19, 0.19, 0.05 (the Graph500 parameters), 2^scale vertices,
  edge_factor * 2^scale draws, vertex labels permuted.
* ``grid_graph(L, seed)``: L x L grid, both directions, plus 0.1% random
  long-range arcs (road-network stand-in).
* ``uniform_batch(...)``: b edges, 80% uniform insertions of vertex pairs and
  20% deletions drawn from the given edge pool.
* ``grid_local_batch(...)``: the same mix, inside one random window.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libdfgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19  # d = 0.05


def build(force: bool = False) -> str:
    """Compiles gen.c into libdfgen.so next to it (if missing or stale)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P32 = ctypes.POINTER(ctypes.c_int32)
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.gen_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, ctypes.c_int,
                                     ctypes.c_int, P32, P32]
            lib.gen_rmat.restype = ctypes.c_int
            lib.gen_filter_below.argtypes = [i64, i32, P32, P32]
            lib.gen_filter_below.restype = i64
            lib.gen_grid_count.argtypes = [i32, i64]
            lib.gen_grid_count.restype = i64
            lib.gen_grid.argtypes = [i32, i64, u64, P32, P32]
            lib.gen_grid.restype = ctypes.c_int
            lib.gen_batch_uniform.argtypes = [i32, i64, i64, u64, P32, P32, i64, ctypes.c_int,
                                              P32, P32, P32, P32]
            lib.gen_batch_uniform.restype = ctypes.c_int
            lib.gen_batch_grid_local.argtypes = [i32, i64, i64, u64, P32, P32, P32, P32, P32]
            lib.gen_batch_grid_local.restype = ctypes.c_int
            lib.gen_uniform.argtypes = [u64, u64, i64, ctypes.POINTER(ctypes.c_double)]
            lib.gen_uniform.restype = None
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def rmat_edges(scale: int, m: int, seed: int, a: float = RMAT_A, b: float = RMAT_B,
               c: float = RMAT_C, permute: bool = True):
    """m raw R-MAT draws over 2^scale labels -> (src, dst) int32 arrays."""
    lib = _load()
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = lib.gen_rmat(scale, m, a, b, c, seed, int(permute), _threads(), _p32(src), _p32(dst))
    if rc != 0:
        raise ValueError(f"gen_rmat failed ({rc})")
    return src, dst


def rmat_graph(scale: int, edge_factor: int, seed: int):
    """(n, src, dst): R-MAT with edge_factor * 2^scale draws (duplicates kept)."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor * n, seed)
    return n, src, dst


def rmat_graph_n(n: int, avg_degree: float, seed: int):
    """R-MAT at a vertex count that need not be a power of two: drawn at the next
    power-of-two scale, draws with an endpoint >= n dropped."""
    scale = max(1, int(np.ceil(np.log2(max(2, n)))))
    m = int(round(avg_degree * n * ((1 << scale) / n) ** 2))
    src, dst = rmat_edges(scale, m, seed)
    k = _load().gen_filter_below(m, n, _p32(src), _p32(dst))
    return n, src[:k].copy(), dst[:k].copy()


def grid_graph(L: int, seed: int, shortcut_frac: float = 1e-3):
    """(n, src, dst): L x L bidirectional grid plus shortcut_frac * arcs random arcs."""
    lib = _load()
    grid_arcs = 4 * L * (L - 1)
    k = int(round(shortcut_frac * grid_arcs))
    m = lib.gen_grid_count(L, k)
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if lib.gen_grid(L, k, seed, _p32(src), _p32(dst)) != 0:
        raise ValueError("gen_grid failed")
    return L * L, src, dst


def split_batch(b: int, ins_frac: float = 0.8):
    n_ins = int(round(b * ins_frac))
    return n_ins, b - n_ins


def uniform_batch(n: int, b: int, seed: int, pool_src: np.ndarray, pool_dst: np.ndarray,
                  ins_frac: float = 0.8):
    """(del_src, del_dst, ins_src, ins_dst) for a batch of b edges."""
    lib = _load()
    n_ins, n_del = split_batch(b, ins_frac)
    out = [np.empty(k, np.int32) for k in (n_ins, n_ins, n_del, n_del)]
    pool_src = np.ascontiguousarray(pool_src, np.int32)
    pool_dst = np.ascontiguousarray(pool_dst, np.int32)
    rc = lib.gen_batch_uniform(n, n_ins, n_del, seed, _p32(pool_src), _p32(pool_dst),
                               len(pool_src), _threads(), *[_p32(x) for x in out])
    if rc != 0:
        raise ValueError("gen_batch_uniform failed")
    ins_src, ins_dst, del_src, del_dst = out
    return del_src, del_dst, ins_src, ins_dst


def grid_local_batch(L: int, b: int, seed: int, ins_frac: float = 0.8):
    """(del_src, del_dst, ins_src, ins_dst) localised in one window of the grid."""
    lib = _load()
    n_ins, n_del = split_batch(b, ins_frac)
    out = [np.empty(k, np.int32) for k in (n_ins, n_ins, n_del, n_del)]
    origin = np.zeros(2, np.int32)
    if lib.gen_batch_grid_local(L, n_ins, n_del, seed, *[_p32(x) for x in out], _p32(origin)) != 0:
        raise ValueError("gen_batch_grid_local failed")
    ins_src, ins_dst, del_src, del_dst = out
    return del_src, del_dst, ins_src, ins_dst


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, np.float64)
    lib.gen_uniform(seed, stream, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def many_graph_specs(count: int, seed: int):
    """Sizes for a many-graph workload: n log-uniform in [1e3, 1e6], average degree
    uniform in [4, 32], batch fraction uniform in [0.001, 0.01]."""
    u = uniform01(seed, 1, 3 * count).reshape(3, count)
    n = np.round(10.0 ** (3.0 + 3.0 * u[0])).astype(np.int64)
    deg = 4.0 + 28.0 * u[1]
    frac = 0.001 + 0.009 * u[2]
    return [(int(n[i]), float(deg[i]), float(frac[i])) for i in range(count)]
