"""CPU oracle for Dynamic Frontier PageRank (plain C, single thread, FP64).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA library (``paper_2407_19562_gb300``) and never imports it.

Functions follow arXiv 2407.19562: Eq. 1 (rank of a vertex), Alg. 3 / Alg. 5
(Static_BB / ND_BB), Alg. 4 / Alg. 6 (Static_LF / ND_LF, one thread), Alg. 1
(DF_BB), Alg. 2 (DF_LF, one thread), the initial marking of Sec. 4.1 and the
batch-update model of Sec. 3.4. See ``oracle.c`` for the readings taken where
the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA = 0.85          # damping factor (Sec. 5.1.2)
TOL = 1e-10           # iteration tolerance, L-inf (Sec. 5.1.2)
TOL_F = TOL / 1000.0  # frontier tolerance (Sec. 4.5)
MAX_ITER = 500        # MAX_ITERATIONS (Sec. 5.1.2)
REF_TOL = 1e-100      # reference ranks (Sec. 5.1.5)


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("processed", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("last_delta", ctypes.c_double),
                ("converged", ctypes.c_int32), ("affected", ctypes.c_int32)]


@dataclass
class Stats:
    iterations: int
    processed: int
    edges: int
    last_delta: float
    converged: bool
    affected: int


def build(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so next to it (if missing or stale)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # DFPR_ORACLE_LIB lets the mutation tests load a copy of the oracle
            # with a planted mistake; it is never set on any other path.
            path = os.environ.get("DFPR_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            vp, i32, i64, dbl, ci = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_int)
            PS = ctypes.POINTER(_Stats)
            lib.orc_graph_build.argtypes = [i32, i64, vp, vp, ci, ctypes.POINTER(vp)]
            lib.orc_graph_apply.argtypes = [vp, i64, vp, vp, i64, vp, vp, ctypes.POINTER(vp), vp]
            lib.orc_graph_free.argtypes = [vp]
            lib.orc_graph_free.restype = None
            lib.orc_graph_n.argtypes = [vp]
            lib.orc_graph_n.restype = i32
            lib.orc_graph_m.argtypes = [vp]
            lib.orc_graph_m.restype = i64
            lib.orc_graph_export.argtypes = [vp, vp, vp, vp, vp]
            lib.orc_graph_export.restype = None
            lib.orc_graph_last_batch.argtypes = [vp, vp, vp, vp, vp, vp]
            lib.orc_graph_last_batch.restype = None
            lib.orc_static_bb.argtypes = [vp, vp, dbl, dbl, ci, ci, vp, PS]
            lib.orc_static_lf.argtypes = [vp, vp, dbl, dbl, ci, vp, PS]
            lib.orc_initial_affected.argtypes = [vp, vp]
            lib.orc_df_bb.argtypes = [vp, vp, dbl, dbl, dbl, ci, vp, PS, vp, ci]
            lib.orc_df_bb_teleport.argtypes = [vp, vp, dbl, dbl, dbl, dbl, ci, vp, PS]
            lib.orc_dangling_mass.argtypes = [vp, vp, vp]
            lib.orc_df_lf.argtypes = [vp, vp, dbl, dbl, dbl, ci, vp, PS]
            lib.orc_sample_rows.argtypes = [i32, i64, vp, vp, ci, i64, vp, vp, i64, vp, vp, ci,
                                            i32, vp, vp, vp, i64]
            lib.orc_sample_rows.restype = i64
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


def _stats(s: _Stats) -> Stats:
    return Stats(int(s.iterations), int(s.processed), int(s.edges), float(s.last_delta),
                 bool(s.converged), int(s.affected))


class Graph:
    """A snapshot G^t: CSR + CSC with sorted unique rows, plus the real changes
    of the batch that produced it."""

    def __init__(self, handle):
        self._h = handle
        self._lib = _load()

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.orc_graph_free(h)

    @classmethod
    def build(cls, n: int, src, dst, self_loops: bool = True) -> "Graph":
        lib = _load()
        src, dst = _i32(src), _i32(dst)
        h = ctypes.c_void_p()
        _check(lib.orc_graph_build(n, len(src), _ptr(src), _ptr(dst), int(self_loops),
                                   ctypes.byref(h)), "graph_build")
        return cls(h)

    def apply(self, del_src, del_dst, ins_src, ins_dst):
        """Returns (G^t, (n_real_del, n_real_ins))."""
        del_src, del_dst, ins_src, ins_dst = map(_i32, (del_src, del_dst, ins_src, ins_dst))
        h = ctypes.c_void_p()
        nr = np.zeros(2, np.int64)
        _check(self._lib.orc_graph_apply(self._h, len(del_src), _ptr(del_src), _ptr(del_dst),
                                         len(ins_src), _ptr(ins_src), _ptr(ins_dst),
                                         ctypes.byref(h), _ptr(nr)), "graph_apply")
        return Graph(h), (int(nr[0]), int(nr[1]))

    @property
    def n(self) -> int:
        return int(self._lib.orc_graph_n(self._h))

    @property
    def m(self) -> int:
        return int(self._lib.orc_graph_m(self._h))

    def csr(self):
        off = np.empty(self.n + 1, np.int64)
        idx = np.empty(self.m, np.int32)
        self._lib.orc_graph_export(self._h, _ptr(off), _ptr(idx), None, None)
        return off, idx

    def csc(self):
        off = np.empty(self.n + 1, np.int64)
        idx = np.empty(self.m, np.int32)
        self._lib.orc_graph_export(self._h, None, None, _ptr(off), _ptr(idx))
        return off, idx

    def last_batch(self):
        """Real changes (del_src, del_dst, ins_src, ins_dst), sorted by (src, dst)."""
        cnt = np.zeros(2, np.int64)
        self._lib.orc_graph_last_batch(self._h, _ptr(cnt), None, None, None, None)
        ds, dd = np.empty(cnt[0], np.int32), np.empty(cnt[0], np.int32)
        is_, id_ = np.empty(cnt[1], np.int32), np.empty(cnt[1], np.int32)
        self._lib.orc_graph_last_batch(self._h, _ptr(cnt), _ptr(ds), _ptr(dd), _ptr(is_),
                                       _ptr(id_))
        return ds, dd, is_, id_

    # --- PageRank ---------------------------------------------------------

    def static_bb(self, R_init=None, alpha=ALPHA, tol=TOL, max_iter=MAX_ITER, dead_end=0):
        """Static_BB (Alg. 3), or ND_BB (Alg. 5) when R_init is given."""
        R = np.empty(self.n, np.float64)
        st = _Stats()
        ri = None if R_init is None else np.ascontiguousarray(R_init, np.float64)
        _check(self._lib.orc_static_bb(self._h, _ptr(ri), alpha, tol, max_iter, dead_end,
                                       _ptr(R), ctypes.byref(st)), "static_bb")
        return R, _stats(st)

    def reference(self, dead_end=0):
        """Reference ranks of Sec. 5.1.5: Static_BB with tol 1e-100, 500 iterations."""
        return self.static_bb(tol=REF_TOL, max_iter=MAX_ITER, dead_end=dead_end)

    def static_lf(self, R_init=None, alpha=ALPHA, tol=TOL, max_iter=MAX_ITER):
        """Static_LF (Alg. 4), or ND_LF (Alg. 6) when R_init is given; one thread."""
        R = np.empty(self.n, np.float64)
        st = _Stats()
        ri = None if R_init is None else np.ascontiguousarray(R_init, np.float64)
        _check(self._lib.orc_static_lf(self._h, _ptr(ri), alpha, tol, max_iter, _ptr(R),
                                       ctypes.byref(st)), "static_lf")
        return R, _stats(st)

    def initial_affected(self) -> np.ndarray:
        va = np.zeros(self.n, np.uint8)
        _check(self._lib.orc_initial_affected(self._h, _ptr(va)), "initial_affected")
        return va

    def df_bb(self, R_prev, alpha=ALPHA, tol=TOL, tol_f=None, max_iter=MAX_ITER, trace=0):
        """DF_BB (Alg. 1). With trace > 0 also returns the affected flags in force
        during iterations 0..trace-1 as a (trace, n) uint8 array."""
        tol_f = tol / 1000.0 if tol_f is None else tol_f
        R = np.empty(self.n, np.float64)
        st = _Stats()
        rp = np.ascontiguousarray(R_prev, np.float64)
        tr = np.zeros((trace, self.n), np.uint8) if trace > 0 else None
        _check(self._lib.orc_df_bb(self._h, _ptr(rp), alpha, tol, tol_f, max_iter, _ptr(R),
                                   ctypes.byref(st), _ptr(tr), trace), "df_bb")
        return (R, _stats(st), tr) if trace > 0 else (R, _stats(st))

    def dangling_mass(self, R):
        """D = sum of R over dead ends (vertices without out-edges)."""
        d = ctypes.c_double()
        r = np.ascontiguousarray(R, np.float64)
        _check(self._lib.orc_dangling_mass(self._h, _ptr(r), ctypes.byref(d)), "dangling_mass")
        return d.value

    def df_bb_teleport(self, R_prev, D_before, alpha=ALPHA, tol=TOL, tol_f=None, max_iter=MAX_ITER):
        """DF_BB (Alg. 1) with the teleport reading of dead ends; D_before is the
        dead-end mass of R_prev on the graph before the batch."""
        tol_f = tol / 1000.0 if tol_f is None else tol_f
        R = np.empty(self.n, np.float64)
        st = _Stats()
        rp = np.ascontiguousarray(R_prev, np.float64)
        _check(self._lib.orc_df_bb_teleport(self._h, _ptr(rp), D_before, alpha, tol, tol_f, max_iter,
                                            _ptr(R), ctypes.byref(st)), "df_bb_teleport")
        return R, _stats(st)

    def df_lf(self, R_prev, alpha=ALPHA, tol=TOL, tol_f=None, max_iter=MAX_ITER):
        """DF_LF (Alg. 2) on one thread, ascending vertex order."""
        tol_f = tol / 1000.0 if tol_f is None else tol_f
        R = np.empty(self.n, np.float64)
        st = _Stats()
        rp = np.ascontiguousarray(R_prev, np.float64)
        _check(self._lib.orc_df_lf(self._h, _ptr(rp), alpha, tol, tol_f, max_iter, _ptr(R),
                                   ctypes.byref(st)), "df_lf")
        return R, _stats(st)


def sample_rows(n, src, dst, which, direction="out", self_loops=True, batch=None, cap=1 << 16):
    """Rows of G^1 = apply(build(src, dst), batch) for the vertices in `which`
    (distinct), computed straight from the raw edges. batch is
    (del_src, del_dst, ins_src, ins_dst) or None. cap: first guess of the
    total row length (grown and retried when short). Returns a list of int32
    arrays."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    which = _i32(which)
    if batch is None:
        e = np.zeros(0, np.int32)
        batch = (e, e, e, e)
    ds, dd, is_, id_ = map(_i32, batch)
    while True:
        off = np.zeros(len(which) + 1, np.int64)
        idx = np.empty(cap, np.int32)
        rc = lib.orc_sample_rows(n, len(src), _ptr(src), _ptr(dst), int(self_loops), len(ds),
                                 _ptr(ds), _ptr(dd), len(is_), _ptr(is_), _ptr(id_),
                                 0 if direction == "out" else 1, len(which), _ptr(which),
                                 _ptr(off), _ptr(idx), cap)
        if rc >= 0:
            return [idx[off[i]:off[i + 1]].copy() for i in range(len(which))]
        if rc != -2 or cap > (1 << 34):
            raise RuntimeError(f"oracle sample_rows failed ({rc})")
        cap *= 4
