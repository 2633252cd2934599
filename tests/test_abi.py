"""The C-ABI library without a GPU: it builds, loads, exports every entry point
include/dfpr.h declares, its structs match the Python binding, and host-side
argument checks return statuses. No compute call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2407_19562_gb300 as dfpr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dfpr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(dfpr_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_builds_and_loads():
    lib = dfpr.load()
    assert os.path.exists(dfpr._build.LIB)
    assert lib.dfpr_version() == 100


def test_every_declared_symbol_is_exported():
    lib = dfpr.load()
    names = declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", dfpr._build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dfpr_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_struct_layout_matches_binding(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "dfpr.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("config %zu\nparams %zu\nstats %zu\n", sizeof(dfpr_graph_config), sizeof(dfpr_params),
         sizeof(dfpr_stats));
  F(dfpr_graph_config, tail_slack); F(dfpr_params, timeout_ms); F(dfpr_params, grid_ctas);
  F(dfpr_params, fault_delay_prob); F(dfpr_params, fault_crash_warps); F(dfpr_params, fault_seed);
  F(dfpr_params, gather_split); F(dfpr_params, mark_split); F(dfpr_params, helping);
  F(dfpr_stats, passes); F(dfpr_stats, residual_linf); F(dfpr_stats, ms);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog),
                           "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).split("\n") if line)
    assert int(got["config"]) == ctypes.sizeof(dfpr.Config)
    assert int(got["params"]) == ctypes.sizeof(dfpr.Params)
    assert int(got["stats"]) == ctypes.sizeof(dfpr.Stats)
    assert int(got["dfpr_graph_config.tail_slack"]) == dfpr.Config.tail_slack.offset
    assert int(got["dfpr_params.timeout_ms"]) == dfpr.Params.timeout_ms.offset
    assert int(got["dfpr_params.grid_ctas"]) == dfpr.Params.grid_ctas.offset
    for f in ("fault_delay_prob", "fault_crash_warps", "fault_seed", "gather_split", "mark_split",
              "helping"):
        assert int(got[f"dfpr_params.{f}"]) == getattr(dfpr.Params, f).offset
    assert int(got["dfpr_stats.passes"]) == dfpr.Stats.passes.offset
    assert int(got["dfpr_stats.residual_linf"]) == dfpr.Stats.residual_linf.offset
    assert int(got["dfpr_stats.ms"]) == dfpr.Stats.ms.offset


def test_defaults_are_the_papers_constants():
    p = dfpr.default_params()
    assert p.alpha == 0.85 and p.tol == 1e-10 and p.max_iter == 500  # Sec. 5.1.2
    assert p.frontier_tol == 0.0  # selects tol / 1000 (Sec. 4.5)
    assert p.mode == dfpr.WORKLIST
    assert p.fault_delay_prob == 0.0 and p.fault_delay_us == 0.0 and p.fault_crash_warps == 0
    assert p.helping == 1  # warps help a stopped warp (Sec. 4.4)
    c = dfpr.default_config()
    assert c.precision == dfpr.FP64 and c.dead_end == dfpr.SELF_LOOPS


def test_host_side_argument_errors():
    lib = dfpr.load()
    src = np.array([0, 1], np.int32)
    # out == NULL, n <= 0, m < 0: rejected before any device work
    assert lib.dfpr_graph_load(4, 2, src.ctypes.data, src.ctypes.data, 0, None, None, None) == dfpr.EINVAL
    h = ctypes.c_void_p()
    assert lib.dfpr_graph_load(0, 2, src.ctypes.data, src.ctypes.data, 0, None, None, ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_graph_load(4, -1, None, None, 0, None, None, ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_graph_load(4, 2, None, None, 0, None, None, ctypes.byref(h)) == dfpr.EINVAL
    assert "n > 0" in dfpr.last_error()
    bad = dfpr.default_config(precision=7)
    assert lib.dfpr_graph_load(4, 2, src.ctypes.data, src.ctypes.data, 0, None, ctypes.byref(bad),
                               ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_apply_batch(None, 0, None, None, 0, None, None, 0, None) == dfpr.EINVAL
    assert lib.dfpr_df_pagerank(None, None, None) == dfpr.EINVAL
    assert lib.dfpr_autotune(None, None, 0, None, None, None) == dfpr.EINVAL
    assert lib.dfpr_get_ranks(None, None, 0) == dfpr.EINVAL
    assert lib.dfpr_graph_free(None) == dfpr.OK
    assert lib.dfpr_set_allocator(dfpr.ALLOC_FN(lambda *a: None), dfpr.FREE_FN(), None) == dfpr.EINVAL


def test_edge_limit_is_checked_before_the_edges_are_read():
    """Edge keys are counted with 32-bit prefix sums, so a graph holds at most
    2^32 - 2 edges, self-loops included. A larger load is rejected before the
    edge arrays are read (the two-element arrays here would not cover it)."""
    lib = dfpr.load()
    h = ctypes.c_void_p()
    src = np.array([0, 1], np.int32)
    limit = (1 << 32) - 2
    n = 4
    # self-loops (the default) add n edges
    assert lib.dfpr_graph_load(n, limit - n + 1, src.ctypes.data, src.ctypes.data, 0, None, None,
                               ctypes.byref(h)) == dfpr.EINVAL
    assert "2^32 - 2 edges" in dfpr.last_error()
    tele = dfpr.default_config(dead_end=dfpr.TELEPORT)
    assert lib.dfpr_graph_load(n, limit + 1, src.ctypes.data, src.ctypes.data, 0, None,
                               ctypes.byref(tele), ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_graph_load(n, 1 << 40, src.ctypes.data, src.ctypes.data, 0, None, None,
                               ctypes.byref(h)) == dfpr.EINVAL
    assert not h.value


def test_binding_rejects_mismatched_arrays():
    with pytest.raises(dfpr.DfprError):
        dfpr._ptr(np.zeros(3, np.int64), np.int32)
    with pytest.raises(dfpr.DfprError):
        dfpr._side(0, 1)


def test_oracle_and_cuda_path_are_independent():
    """Neither side imports, includes or links the other."""
    pkg = os.path.join(ROOT, "paper_2407_19562_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", text), f"{f} mentions the oracle"
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "import paper_2407_19562_gb300" not in text and "dfpr.h" not in text


def test_graph_set_host_side_checks():
    lib = dfpr.load()
    h = ctypes.c_void_p()
    src = np.array([0, 1], np.int32)
    bad0 = np.array([1, 5], np.int32)       # offsets must start at 0
    flat = np.array([0, 4, 4], np.int32)    # every graph needs a vertex
    for off in (bad0, flat):
        assert lib.dfpr_graph_load_parts(len(off) - 1, off.ctypes.data, 2, src.ctypes.data,
                                         src.ctypes.data, 0, None, None, ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_graph_load_parts(0, bad0.ctypes.data, 0, None, None, 0, None, None,
                                     ctypes.byref(h)) == dfpr.EINVAL
    tele = dfpr.default_config(dead_end=dfpr.TELEPORT)
    ok = np.array([0, 2, 4], np.int32)
    assert lib.dfpr_graph_load_parts(2, ok.ctypes.data, 2, src.ctypes.data, src.ctypes.data, 0,
                                     None, ctypes.byref(tele), ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_get_part_times(None, None) == dfpr.EINVAL


def test_server_host_side_checks():
    lib = dfpr.load()
    h = ctypes.c_void_p()
    assert lib.dfpr_server_create(None, None, 4, 0.5, ctypes.byref(h)) == dfpr.EINVAL
    assert lib.dfpr_server_submit(None, 0, 0, None, None, 0, None, None, None) == dfpr.EINVAL
    assert lib.dfpr_server_wait(None, 1, None) == dfpr.EINVAL
    assert lib.dfpr_server_drain(None) == dfpr.EINVAL
    assert lib.dfpr_server_destroy(None) == dfpr.OK
