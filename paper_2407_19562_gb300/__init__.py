"""Python binding of libdfpr (Dynamic Frontier PageRank on GB300, sm_103a).

Argument marshalling only: every function forwards to the C entry point of the
same name in ``include/dfpr.h`` (``graph_load`` -> ``dfpr_graph_load`` ...).
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); all arrays
of one call must live on the same side. There is no CPU fallback: if the CUDA
library cannot be built or loaded, ``load()`` raises.

Hard failures (bad arguments, CUDA errors, out of memory, busy graph) raise
``DfprError``. A rank computation stopped by its iteration cap or time budget
returns its stats with ``status`` set to ``ENOTCONV`` / ``ETIMEOUT``; the
ranks are valid but not converged.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

__all__ = [
    "DfprError", "Config", "Params", "Stats", "Graph", "load", "version", "last_error",
    "kernel_launches",
    "default_config", "default_params", "graph_load", "graph_free", "graph_info",
    "graph_set_stream", "apply_batch", "df_pagerank", "nd_pagerank", "static_pagerank",
    "get_ranks", "set_ranks", "residual", "set_capture", "capture_info", "get_csr", "get_csc", "initial_affected", "set_allocator",
    "graph_load_parts", "get_part_times", "autotune", "autotune_plans", "Server", "RequestInfo", "server_create",
    "use_torch_allocator", "OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONV", "ETIMEOUT", "EBUSY",
    "FP64", "FP32", "SELF_LOOPS", "TELEPORT", "WORKLIST", "ROUND", "JACOBI",
]

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT, EBUSY = range(7)
FP64, FP32 = 0, 1
SELF_LOOPS, TELEPORT = 0, 1
WORKLIST, ROUND, JACOBI = 0, 1, 2
_STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONV", "ETIMEOUT", "EBUSY"]


class DfprError(RuntimeError):
    """A failed library call: .status is the dfpr_status code; the message is
    the library's dfpr_last_error() text."""
    def __init__(self, status: int, where: str, message: str):
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")
        self.status = status


class Config(ctypes.Structure):
    """dfpr_graph_config: options fixed when a graph is loaded."""
    _fields_ = [("precision", ctypes.c_int32), ("dead_end", ctypes.c_int32),
                ("row_slack", ctypes.c_double), ("min_slack", ctypes.c_int32),
                ("reorder", ctypes.c_int32), ("tail_slack", ctypes.c_double)]


class Params(ctypes.Structure):
    """dfpr_params: parameters of one rank computation (see default_params)."""
    _fields_ = [("alpha", ctypes.c_double), ("tol", ctypes.c_double),
                ("frontier_tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("normalize", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("timeout_ms", ctypes.c_double),
                ("fault_delay_prob", ctypes.c_double), ("fault_delay_us", ctypes.c_double),
                ("fault_crash_warps", ctypes.c_int32), ("fault_seed", ctypes.c_uint32),
                ("gather_split", ctypes.c_int32), ("mark_split", ctypes.c_int32),
                ("helping", ctypes.c_int32)]


class Stats(ctypes.Structure):
    """dfpr_stats: counters of one call; .status holds the call's dfpr_status."""
    _fields_ = [("processed", ctypes.c_int64), ("edges_gathered", ctypes.c_int64),
                ("expansions", ctypes.c_int64), ("edges_marked", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("affected", ctypes.c_int64),
                ("passes", ctypes.c_int32), ("status", ctypes.c_int32),
                ("residual_linf", ctypes.c_double), ("rank_sum", ctypes.c_double),
                ("ms", ctypes.c_double), ("batches", ctypes.c_int64),
                ("tokens", ctypes.c_int64), ("jobs", ctypes.c_int64),
                ("phase_cycles", ctypes.c_int64 * 5)]

    PHASES = ("idle", "claim", "gather", "expand", "finish")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_cycles"}
        d["phase_cycles"] = dict(zip(self.PHASES, list(self.phase_cycles)))
        return d


class RequestInfo(ctypes.Structure):
    """dfpr_request_info: outcome and host-clock times of one served request."""
    _fields_ = [("status", ctypes.c_int32), ("cycle_requests", ctypes.c_int32),
                ("cycle", ctypes.c_int64), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)

_lib = None
_lock = threading.Lock()
_keep = []  # callbacks installed with set_allocator


def load():
    """Builds (if stale) and loads libdfpr.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp, i32, i64, ci = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
        st = ctypes.c_int
        sig = {
            "dfpr_default_config": (None, [ctypes.POINTER(Config)]),
            "dfpr_default_params": (None, [ctypes.POINTER(Params)]),
            "dfpr_graph_load": (st, [i32, i64, vp, vp, ci, vp, ctypes.POINTER(Config),
                                     ctypes.POINTER(vp)]),
            "dfpr_graph_load_parts": (st, [i32, vp, i64, vp, vp, ci, vp, ctypes.POINTER(Config),
                                           ctypes.POINTER(vp)]),
            "dfpr_graph_parts": (st, [vp, ctypes.POINTER(i32)]),
            "dfpr_get_part_times": (st, [vp, vp]),
            "dfpr_server_create": (st, [vp, ctypes.POINTER(Params), i32, ctypes.c_double,
                                        ctypes.POINTER(vp)]),
            "dfpr_server_create_units": (st, [i32, vp, ctypes.POINTER(Params), i32,
                                              ctypes.c_double, i32, ctypes.POINTER(vp)]),
            "dfpr_server_submit": (st, [vp, i32, i64, vp, vp, i64, vp, vp, ctypes.POINTER(i64)]),
            "dfpr_server_wait": (st, [vp, i64, ctypes.POINTER(RequestInfo)]),
            "dfpr_server_drain": (st, [vp]),
            "dfpr_server_destroy": (st, [vp]),
            "dfpr_graph_free": (st, [vp]),
            "dfpr_graph_set_stream": (st, [vp, vp]),
            "dfpr_graph_info": (st, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                     ctypes.POINTER(i32)]),
            "dfpr_apply_batch": (st, [vp, i64, vp, vp, i64, vp, vp, ci, ctypes.POINTER(i64)]),
            "dfpr_df_pagerank": (st, [vp, ctypes.POINTER(Params), ctypes.POINTER(Stats)]),
            "dfpr_autotune": (st, [vp, ctypes.POINTER(Params), i32, vp, vp, ctypes.POINTER(Stats)]),
            "dfpr_nd_pagerank": (st, [vp, ctypes.POINTER(Params), ctypes.POINTER(Stats)]),
            "dfpr_static_pagerank": (st, [vp, ctypes.POINTER(Params), ctypes.POINTER(Stats)]),
            "dfpr_get_ranks": (st, [vp, vp, ci]),
            "dfpr_set_ranks": (st, [vp, vp, ci]),
            "dfpr_get_csr": (st, [vp, vp, vp, ci]),
            "dfpr_get_csc": (st, [vp, vp, vp, ci]),
            "dfpr_initial_affected": (st, [vp, vp, ci, ctypes.POINTER(i64)]),
            "dfpr_set_allocator": (st, [ALLOC_FN, FREE_FN, vp]),
            "dfpr_last_error": (ctypes.c_char_p, []),
            "dfpr_version": (i32, []),
            "dfpr_kernel_launches": (i64, []),
            "dfpr_autotune_plans": (st, [vp, ctypes.POINTER(Params), i32, vp, ctypes.POINTER(i32),
                                         vp, vp, ctypes.POINTER(Stats)]),
            "dfpr_graph_set_capture": (st, [vp, i32]),
            "dfpr_graph_capture_info": (st, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "dfpr_residual": (st, [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
            "dfpr_static_pagerank_noalloc": (st, [i32, vp, vp, vp, ctypes.c_double,
                                                  ctypes.c_double, i32, vp,
                                                  ctypes.POINTER(i32), vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def version() -> int:
    """dfpr_version: the library's ABI version."""
    return int(load().dfpr_version())


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().dfpr_kernel_launches())


def last_error() -> str:
    """dfpr_last_error: this thread's last error message."""
    return (load().dfpr_last_error() or b"").decode(errors="replace")


def _check(rc: int, where: str):
    if rc != OK:
        raise DfprError(rc, where, last_error())


def default_config(**kw) -> Config:
    """dfpr_default_config, with any field overridden by keyword."""
    c = Config()
    load().dfpr_default_config(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_params(**kw) -> Params:
    """dfpr_default_params (the paper's constants), with any field overridden by
    keyword."""
    p = Params()
    load().dfpr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# --------------------------------------------------------------------------
# array marshalling
# --------------------------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype, n_expected=None, name="array"):
    """(pointer, length, on_device) of a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        import torch
        tdt = {np.int32: torch.int32, np.float64: torch.float64, np.int64: torch.int64,
               np.uint8: torch.uint8}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise DfprError(EINVAL, name, f"need a contiguous {tdt} tensor")
        n = x.numel()
        on_dev = 1 if x.is_cuda else 0
        ptr = x.data_ptr()
    else:
        if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
            raise DfprError(EINVAL, name, f"need a contiguous numpy {np.dtype(dtype)} array")
        n = x.size
        on_dev = 0
        ptr = x.ctypes.data
    if n_expected is not None and n != n_expected:
        raise DfprError(EINVAL, name, f"expected {n_expected} elements, got {n}")
    return (ptr if n else None), n, on_dev


def _side(*sides):
    s = {x for x in sides if x is not None}
    if len(s) > 1:
        raise DfprError(EINVAL, "arrays", "all arrays of one call must be on the same side")
    return s.pop() if s else 0


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # noqa: BLE001 - torch is optional plumbing
        pass
    return None


# --------------------------------------------------------------------------
# graph handle
# --------------------------------------------------------------------------

class Graph:
    """Owns a dfpr_graph*; freed by graph_free() or on garbage collection."""

    def __init__(self, handle: int, n: int):
        self._h = handle
        self.n = n

    @property
    def handle(self):
        if not self._h:
            raise DfprError(EINVAL, "graph", "graph was freed")
        return self._h

    def free(self):
        h = self._h
        if h:
            _check(load().dfpr_graph_free(h), "graph_free")  # EBUSY keeps the handle
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    # convenience methods mirroring the module functions
    def apply_batch(self, *a, **k):
        return apply_batch(self, *a, **k)

    def df_pagerank(self, *a, **k):
        return df_pagerank(self, *a, **k)

    def nd_pagerank(self, *a, **k):
        return nd_pagerank(self, *a, **k)

    def autotune(self, *a, **k):
        return autotune(self, *a, **k)

    def autotune_plans(self, *a, **k):
        return autotune_plans(self, *a, **k)

    def static_pagerank(self, *a, **k):
        return static_pagerank(self, *a, **k)

    def get_ranks(self, *a, **k):
        return get_ranks(self, *a, **k)

    def set_ranks(self, *a, **k):
        return set_ranks(self, *a, **k)

    def residual(self, *a, **k):
        return residual(self, *a, **k)

    def set_capture(self, *a, **k):
        return set_capture(self, *a, **k)

    def capture_info(self):
        return capture_info(self)

    def get_csr(self, *a, **k):
        return get_csr(self, *a, **k)

    def get_csc(self, *a, **k):
        return get_csc(self, *a, **k)

    def initial_affected(self, *a, **k):
        return initial_affected(self, *a, **k)

    def info(self):
        return graph_info(self)


def graph_load(n: int, src, dst, config: Config | None = None, stream="torch") -> Graph:
    """dfpr_graph_load. stream: a cudaStream_t (int), None for a library-owned
    stream, or "torch" for torch's current stream when torch has initialised CUDA."""
    lib = load()
    ps, ms, ds = _ptr(src, np.int32, name="src")
    pd, md, dd = _ptr(dst, np.int32, name="dst")
    if ms != md:
        raise DfprError(EINVAL, "graph_load", "src and dst lengths differ")
    on_dev = _side(ds, dd)
    s = _torch_stream() if stream == "torch" else stream
    h = ctypes.c_void_p()
    _check(lib.dfpr_graph_load(int(n), ms, ps, pd, on_dev, s,
                               ctypes.byref(config) if config is not None else None,
                               ctypes.byref(h)), "graph_load")
    return Graph(h.value, int(n))


def graph_load_parts(vertex_offsets, src, dst, config: Config | None = None,
                     stream="torch") -> Graph:
    """dfpr_graph_load_parts: k graphs as one set; vertex_offsets has k + 1
    entries and src/dst use global ids."""
    lib = load()
    off = np.ascontiguousarray(vertex_offsets, dtype=np.int32)
    ps, ms, ds = _ptr(src, np.int32, name="src")
    pd, md, dd = _ptr(dst, np.int32, name="dst")
    if ms != md:
        raise DfprError(EINVAL, "graph_load_parts", "src and dst lengths differ")
    on_dev = _side(ds, dd)
    s = _torch_stream() if stream == "torch" else stream
    h = ctypes.c_void_p()
    _check(lib.dfpr_graph_load_parts(len(off) - 1, off.ctypes.data, ms, ps, pd, on_dev, s,
                                     ctypes.byref(config) if config is not None else None,
                                     ctypes.byref(h)), "graph_load_parts")
    g = Graph(h.value, int(off[-1]))
    g.parts = len(off) - 1
    return g


def get_part_times(g: Graph) -> np.ndarray:
    """dfpr_get_part_times: per-graph completion ms of the last worklist update."""
    k = ctypes.c_int32()
    _check(load().dfpr_graph_parts(g.handle, ctypes.byref(k)), "graph_parts")
    out = np.zeros(k.value, np.float64)
    _check(load().dfpr_get_part_times(g.handle, out.ctypes.data), "get_part_times")
    return out


def graph_free(g: Graph):
    """dfpr_graph_free (EBUSY while another call on g runs)."""
    g.free()


def graph_set_stream(g: Graph, stream):
    """dfpr_graph_set_stream: later calls on g run on `stream` (a cudaStream_t;
    None: a new stream of the library's)."""
    _check(load().dfpr_graph_set_stream(g.handle, stream), "graph_set_stream")


def graph_info(g: Graph):
    """dfpr_graph_info -> {"n", "m" (edges with self-loops), "device"}."""
    n, m, dev = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(load().dfpr_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(dev)),
           "graph_info")
    return {"n": n.value, "m": m.value, "device": dev.value}


def apply_batch(g: Graph, del_src, del_dst, ins_src, ins_dst):
    """dfpr_apply_batch -> (real deletions, real insertions)."""
    a = [_ptr(x, np.int32, name=nm) for x, nm in
         ((del_src, "del_src"), (del_dst, "del_dst"), (ins_src, "ins_src"), (ins_dst, "ins_dst"))]
    if a[0][1] != a[1][1] or a[2][1] != a[3][1]:
        raise DfprError(EINVAL, "apply_batch", "source and target lengths differ")
    on_dev = _side(*(x[2] for x in a))
    out = (ctypes.c_int64 * 2)()
    _check(load().dfpr_apply_batch(g.handle, a[0][1], a[0][0], a[1][0], a[2][1], a[2][0],
                                   a[3][0], on_dev, out), "apply_batch")
    return int(out[0]), int(out[1])


def _run(fn, where, g, params):
    st = Stats()
    p = params if params is not None else default_params()
    rc = fn(g.handle, ctypes.byref(p), ctypes.byref(st))
    if rc not in (OK, ENOTCONV, ETIMEOUT):
        _check(rc, where)
    st.status = rc
    return st


def df_pagerank(g: Graph, params: Params | None = None) -> Stats:
    """dfpr_df_pagerank: the DF update for the pending changes. ENOTCONV and
    ETIMEOUT come back in Stats.status (ranks valid, not converged); other
    failures raise DfprError."""
    return _run(load().dfpr_df_pagerank, "df_pagerank", g, params)


def autotune(g: Graph, params: Params | None = None, candidates=None):
    """dfpr_autotune: times the pending update under each (gather_split,
    mark_split) pair and leaves it applied with the fastest one. Returns
    (tuned Params, trial times in ms, Stats of the final update)."""
    p = Params.from_buffer_copy(params if params is not None else default_params())
    if candidates is None:
        k, cand, n_trials = 0, None, 4
    else:
        arr = np.ascontiguousarray(np.asarray(candidates, np.int32).reshape(-1, 2))
        k, cand, n_trials = len(arr), arr, len(arr)
    trials = np.zeros(n_trials, np.float64)
    st = Stats()
    rc = load().dfpr_autotune(g.handle, ctypes.byref(p), k,
                              cand.ctypes.data if cand is not None else None,
                              trials.ctypes.data, ctypes.byref(st))
    if rc not in (OK, ENOTCONV, ETIMEOUT):
        _check(rc, "autotune")
    st.status = rc
    return p, trials, st


def autotune_plans(g: Graph, params: Params | None = None, plans=None):
    """dfpr_autotune_plans: times the pending update under each plan (mode,
    grid_ctas, gather_split, mark_split) and leaves it applied with the
    fastest. plans None: the library's built-in set. Returns (tuned Params,
    the plans timed as an (k, 4) int32 array, their times in ms, Stats of the
    final update)."""
    p = Params.from_buffer_copy(params if params is not None else default_params())
    if plans is None:
        k, arr = 0, None
    else:
        arr = np.ascontiguousarray(np.asarray(plans, np.int32).reshape(-1, 4))
        k = len(arr)
    cap = max(k, 8)
    run = ctypes.c_int32()
    plans_run = np.zeros((cap, 4), np.int32)
    trials = np.zeros(cap, np.float64)
    st = Stats()
    rc = load().dfpr_autotune_plans(g.handle, ctypes.byref(p), k,
                                    arr.ctypes.data if arr is not None else None,
                                    ctypes.byref(run), plans_run.ctypes.data, trials.ctypes.data,
                                    ctypes.byref(st))
    if rc not in (OK, ENOTCONV, ETIMEOUT):
        _check(rc, "autotune_plans")
    st.status = rc
    r = run.value
    return p, plans_run[:r].copy(), trials[:r].copy(), st


def nd_pagerank(g: Graph, params: Params | None = None) -> Stats:
    """dfpr_nd_pagerank: naive-dynamic update from the current ranks."""
    return _run(load().dfpr_nd_pagerank, "nd_pagerank", g, params)


def static_pagerank(g: Graph, params: Params | None = None) -> Stats:
    """dfpr_static_pagerank: ranks from 1/n on the current graph."""
    return _run(load().dfpr_static_pagerank, "static_pagerank", g, params)


def get_ranks(g: Graph, out=None):
    """dfpr_get_ranks into `out` (numpy float64 or torch float64, host or CUDA);
    returns a new numpy array when out is None."""
    if out is None:
        out = np.empty(g.n, np.float64)
    p, _, dev = _ptr(out, np.float64, g.n, "out")
    _check(load().dfpr_get_ranks(g.handle, p, dev), "get_ranks")
    return out


def set_capture(g: Graph, enable: bool = True):
    """dfpr_graph_set_capture: replay the worklist DF update's device work from a
    CUDA graph (captured on the first call), or go back to eager launches."""
    _check(load().dfpr_graph_set_capture(g.handle, 1 if enable else 0), "set_capture")


def capture_info(g: Graph):
    """dfpr_graph_capture_info -> (captures made, replays launched)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().dfpr_graph_capture_info(g.handle, ctypes.byref(a), ctypes.byref(b)), "capture_info")
    return a.value, b.value


def residual(g: Graph, alpha: float = 0.85):
    """dfpr_residual -> (max_v |Eq. 1 (v) - R[v]|, the same relative to R[v]),
    both computed in FP64 from the stored ranks."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().dfpr_residual(g.handle, float(alpha), ctypes.byref(a), ctypes.byref(b)), "residual")
    return a.value, b.value


def set_ranks(g: Graph, ranks):
    """dfpr_set_ranks from a float64 array (numpy, or torch on the host or the
    graph's device)."""
    p, _, dev = _ptr(ranks, np.float64, g.n, "ranks")
    _check(load().dfpr_set_ranks(g.handle, p, dev), "set_ranks")


def _export(fn, where, g, offsets, idx):
    info = graph_info(g)
    if offsets is None:
        offsets = np.empty(info["n"] + 1, np.int64)
    if idx is None:
        idx = np.empty(max(info["m"], 1), np.int32)[:info["m"]]
    po, _, d1 = _ptr(offsets, np.int64, info["n"] + 1, "offsets")
    pi, _, d2 = _ptr(idx, np.int32, info["m"], "idx")
    if pi is None:  # empty graph: give a valid pointer
        keep = np.empty(1, np.int32)
        pi = keep.ctypes.data
    _check(fn(g.handle, po, pi, _side(d1, d2)), where)
    return offsets, idx


def get_csr(g: Graph, offsets=None, idx=None):
    """dfpr_get_csr -> (offsets int64[n + 1], idx int32[m]), caller ids; writes
    into the given arrays (host or device) when passed."""
    return _export(load().dfpr_get_csr, "get_csr", g, offsets, idx)


def get_csc(g: Graph, offsets=None, idx=None):
    """dfpr_get_csc -> (offsets int64[n + 1], idx int32[m]), caller ids."""
    return _export(load().dfpr_get_csc, "get_csc", g, offsets, idx)


def initial_affected(g: Graph, out=None):
    """dfpr_initial_affected -> (flags uint8[n], count)."""
    if out is None:
        out = np.zeros(g.n, np.uint8)
    p, _, dev = _ptr(out, np.uint8, g.n, "out")
    cnt = ctypes.c_int64()
    _check(load().dfpr_initial_affected(g.handle, p, dev, ctypes.byref(cnt)), "initial_affected")
    return out, int(cnt.value)


class Server:
    """dfpr_server_*: native worker threads serving update requests on one or
    more resident units (graphs or sets). submit() queues one graph's batch
    (host arrays, local ids; parts numbered over the units in order) and
    returns a request id; wait() blocks until the update that served it is done."""

    def __init__(self, handle: int, units):
        self._h = handle
        self.units = list(units)
        self.graph = self.units[0]

    def submit(self, part, del_src, del_dst, ins_src, ins_dst) -> int:
        """dfpr_server_submit: queues one batch for graph `part` -> request id."""
        a = [np.ascontiguousarray(x, np.int32) for x in (del_src, del_dst, ins_src, ins_dst)]
        if len(a[0]) != len(a[1]) or len(a[2]) != len(a[3]):
            raise DfprError(EINVAL, "server_submit", "source and target lengths differ")
        rid = ctypes.c_int64()
        _check(load().dfpr_server_submit(self._h, int(part), len(a[0]), a[0].ctypes.data,
                                         a[1].ctypes.data, len(a[2]), a[2].ctypes.data,
                                         a[3].ctypes.data, ctypes.byref(rid)), "server_submit")
        return int(rid.value)

    def wait(self, request_id: int) -> RequestInfo:
        """dfpr_server_wait: blocks until the update that served the request finished."""
        info = RequestInfo()
        _check(load().dfpr_server_wait(self._h, int(request_id), ctypes.byref(info)), "server_wait")
        return info

    def drain(self):
        """dfpr_server_drain: blocks until every queued request is served."""
        _check(load().dfpr_server_drain(self._h), "server_drain")

    def destroy(self):
        """dfpr_server_destroy: drains, stops the worker threads and frees the
        server (the units stay)."""
        h, self._h = self._h, None
        if h:
            _check(load().dfpr_server_destroy(h), "server_destroy")

    def __del__(self):
        try:
            self.destroy()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def server_create(g, params: Params | None = None, max_slots: int = 64,
                  mem_fraction: float = 0.5, grid_share: int = 0) -> Server:
    """dfpr_server_create_units over g (a Graph, or a list of Graphs each with
    its own stream): a unit's worker admits its queued requests whenever the
    unit is idle, at most max_slots in flight over the server and while their
    batches fit mem_fraction of the device's free memory, and updates them in
    one launch; units update concurrently. grid_share > 0 caps each launch at
    that many CTAs so that several units' launches fit on the GPU together."""
    units = list(g) if isinstance(g, (list, tuple)) else [g]
    arr = (ctypes.c_void_p * len(units))(*[u.handle for u in units])
    h = ctypes.c_void_p()
    _check(load().dfpr_server_create_units(len(units), arr,
                                           ctypes.byref(params) if params is not None else None,
                                           int(max_slots), float(mem_fraction), int(grid_share),
                                           ctypes.byref(h)),
           "server_create")
    return Server(h.value, units)


def set_allocator(alloc=None, free=None, ctx=None):
    """dfpr_set_allocator with Python callables alloc(bytes, stream) -> int and
    free(ptr, bytes, stream); None, None restores cudaMalloc."""
    lib = load()
    if alloc is None and free is None:
        _check(lib.dfpr_set_allocator(ALLOC_FN(), FREE_FN(), None), "set_allocator")
        return
    a = ALLOC_FN(lambda nbytes, stream, _c: alloc(nbytes, stream) or None)
    f = FREE_FN(lambda ptr, nbytes, stream, _c: free(ptr, nbytes, stream))
    _keep.extend([a, f])
    _check(lib.dfpr_set_allocator(a, f, ctx), "set_allocator")


def use_torch_allocator():
    """Routes the library's device allocations through torch's caching allocator."""
    import torch

    def alloc(nbytes, stream):
        try:
            s = torch.cuda.ExternalStream(stream) if stream else None
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=s)
        except Exception:  # noqa: BLE001 - reported to the library as NULL
            return None

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)
