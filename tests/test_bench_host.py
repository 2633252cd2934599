"""Host-side pieces of bench.py that shape its JSON line, checked on the CPU:
the oracle sample and its scale factor, the baseline entry, the byte model
of the roofline and the guard that retires a traffic figure once the kernel
code changes."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sample_is_the_workload_at_a_smaller_size():
    b = load_bench()
    s, f = b.sample_spec(b.WORKLOADS["rmat24"], 18)
    assert (s["scale"], s["edge_factor"], s["seed"], f) == (18, 16, 3, 64.0)
    s, f = b.sample_spec(b.WORKLOADS["rmat24e4"], 18)
    assert (s["scale"], s["edge_factor"], f) == (18, 4, 64.0)      # same edge factor
    s, f = b.sample_spec(b.WORKLOADS["grid4096"], 18)
    assert (s["L"], f) == (512, 64.0)                               # (4096 / 512)^2
    s, f = b.sample_spec(b.WORKLOADS["rmat14"], 18)
    assert (s["scale"], f) == (14, 1.0)                             # never larger than the workload


def test_baseline_entry_scales_the_sample():
    b = load_bench()
    e = b.cpu_baseline_entry([100.0, 140.0], 64.0, "desc")
    assert e["value"] == 120.0 * 64.0 and e["sample_ms_per_batch"] == 120.0
    assert (e["kind"], e["cores"], e["unit"], e["scale_factor"]) == ("oracle", 1, b.UNIT, 64.0)


def test_algorithmic_bytes_per_work_unit():
    b = load_bench()
    one = dict(processed=0, edges_gathered=0, expansions=0, edges_marked=0, pushes=0)
    per = {"processed": (44, 32), "edges_gathered": (12, 8), "expansions": (16, 16),
           "edges_marked": (8, 8), "pushes": (8, 8)}
    for k, (b64, b32) in per.items():
        st = dict(one, **{k: 1})
        assert b.algorithmic_bytes(st, 8) == b64, k
        assert b.algorithmic_bytes(st, 4) == b32, k


def test_traffic_figure_retires_with_the_kernel_code(monkeypatch):
    b = load_bench()
    key = ("rmat24-batch0.0001", "fp64", "worklist")
    digest, traffic, alg = b.MEASURED_TRAFFIC[key]  # the recorded capture's format
    assert len(digest) == 16 and traffic >= 0 and alg >= 0
    assert len(b.kernel_source_hash()) == 16
    monkeypatch.setitem(b.MEASURED_TRAFFIC, key, ("ab" * 8, 100e9, 80e9))
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "ab" * 8)
    assert b.measured_traffic(*key) == (100e9, 80e9)  # the sources the capture ran
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "0" * 16)
    assert b.measured_traffic(*key) is None     # changed code: no stale figure
    assert b.measured_traffic("rmat20-batch0.0001", "fp64", "worklist") is None


def test_working_set_and_l2_flag():
    import torch
    b = load_bench()
    # R-MAT scale 14 (the small workload) sits far inside a 126 MB L2; scale 24 does not
    assert b.working_set_bytes(16384, 278_000, 8) < 4e6
    assert b.working_set_bytes(16_777_216, 280_209_127, 8) > 3e9
    assert b.working_set_bytes(10, 100, 4) == 8 * 100 + 10 * (32 + 16) + 10 // 4
    if not torch.cuda.is_available():
        assert b.l2_bytes(0) == 0       # unknown without a GPU, never an exception
