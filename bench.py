#!/usr/bin/env python3
"""Benchmark of the Dynamic Frontier PageRank update on GB300.

One step = one batch through the whole hot path: dfpr_apply_batch (CSR/CSC
update, real-change extraction) + dfpr_df_pagerank (marking, persistent
frontier iteration). Default workload: R-MAT scale 24 (16.7M vertices, 268M
edge draws, a, b, c, d = .57, .19, .19, .05), batches of 1e-4 |E| edges
(80% uniform insertions, 20% deletions of existing edges), FP64 ranks,
alpha = 0.85, tau = 1e-10, tau_f = tau / 1000. Ranks start from a converged
static PageRank (untimed). Each timed step applies a new batch to the
evolving graph; L2 is flushed (256 MiB write) between steps outside the
events.

Prints one JSON line (rank 0). --impl reference times the CPU oracle (one
core) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "DF update ms/batch (apply_batch + df_pagerank)"
UNIT = "ms/batch"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["rmat24", "rmat20", "rmat24e4", "rmat14", "grid4096", "many256",
                                           "serve8", "faults", "sweep", "stream"], default="rmat24")
    ap.add_argument("--graph", choices=["rmat24", "rmat20", "rmat24e4", "grid4096"], default="rmat24",
                    help="sweep: the graph")
    ap.add_argument("--requests", type=int, default=300, help="serve8: requests per load point")
    ap.add_argument("--units", type=int, default=2,
                    help="serve8: continuous form over this many units (sets of graphs)")
    ap.add_argument("--share-div", type=int, default=2,
                    help="serve8: continuous launches are capped at 1/share-div of a wave")
    ap.add_argument("--graphs", type=int, default=256, help="many256: number of graphs")
    ap.add_argument("--autotune", action="store_true",
                    help="many256: pick the set's schedule, grid and split thresholds with "
                         "dfpr_autotune_plans on the first (warm-up) step")
    ap.add_argument("--batch-frac", type=float, default=1e-4)
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--mode", choices=["worklist", "round", "jacobi"], default="worklist")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="rmat24: skip the FP32, grid, many-graph and serving keys of the line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-scale", type=int, default=18)
    ap.add_argument("--timeout-ms", type=float, default=60000.0)
    return ap.parse_args()


WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, edge_factor=16, seed=3),
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, seed=3),
    # profile case: vectors larger than L2 (n = 16.8M) but ~2 GB on the device
    "rmat24e4": dict(kind="rmat", scale=24, edge_factor=4, seed=3),
    "rmat14": dict(kind="rmat", scale=14, edge_factor=16, seed=1),
    "grid4096": dict(kind="grid", L=4096, seed=4),
}


def make_graph(spec):
    if spec["kind"] == "rmat":
        return workloads.rmat_graph(spec["scale"], spec["edge_factor"], spec["seed"])
    return workloads.grid_graph(spec["L"], spec["seed"])


def make_batch(spec, n, src, dst, b, seed):
    if spec["kind"] == "rmat":
        return workloads.uniform_batch(n, b, seed, src, dst)
    return workloads.grid_local_batch(spec["L"], b, seed)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic bytes of the persistent DF kernel (FP64 / FP32 ranks)
# --------------------------------------------------------------------------

def working_set_bytes(n: int, m: int, s_r: int) -> int:
    """Device bytes an update can touch: in- and out-row ids (4 B per edge
    each), both row descriptors (16 B each per vertex), rank and contribution
    (s_R each), the per-vertex X + epoch record (2 s_R) and the 2-bit
    states."""
    return 8 * m + n * (32 + 4 * s_r) + n // 4


def l2_bytes(dev) -> int:
    """L2 size of the device (0 when the runtime does not report it)."""
    import torch
    try:
        return int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 0)
    except Exception:  # noqa: BLE001 - reported as unknown
        return 0


def algorithmic_bytes(st, s_r: int) -> float:
    """Bytes the method must move for the counted work, whatever the layout:
    per recomputed vertex: in-row offset and degree (16 B), out-degree (4 B),
    own rank read, rank and contribution writes (3 s_R); per gathered in-edge:
    id (4 B) + contribution (s_R); per expansion: the out-row offset and degree
    (16 B); per marked out-edge: id (4 B) + flag word RMW (4 B); per queue
    insertion: slot write + read (8 B)."""
    return (st["processed"] * (20 + 3 * s_r) + st["edges_gathered"] * (4 + s_r)
            + st["expansions"] * 16 + st["edges_marked"] * 8 + st["pushes"] * 8)


def phase_share(stats):
    """Share of the persistent kernel's warp-cycles per phase (summed over steps)."""
    tot = {}
    for s in stats:
        for k, v in s.get("phase_cycles", {}).items():
            tot[k] = tot.get(k, 0) + v
    all_ = sum(tot.values()) or 1
    return {k: round(v / all_, 4) for k, v in tot.items()}


def host_residual(R, in_off, in_idx, part_off=None, alpha=0.85, sample=200_000, seed=0):
    """Largest |Eq. 1 (v) - R[v]| and |Eq. 1 (v) - R[v]| / R[v] over sampled
    vertices, evaluated with numpy in FP64 from exported in-rows (caller ids)
    and ranks; out-degrees are counted from the in-rows. part_off: vertex
    offsets of the graphs of a set (each graph its own n in the teleport term)."""
    n = len(R)
    outdeg = np.bincount(in_idx, minlength=n).astype(np.float64)
    contrib = np.where(outdeg > 0, R / np.maximum(outdeg, 1.0), 0.0)
    rng = np.random.default_rng(seed)
    v = np.unique(rng.integers(0, n, size=min(sample, n)))
    lo, hi = in_off[v], in_off[v + 1]
    lens = (hi - lo).astype(np.int64)
    idx = np.repeat(lo - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + np.arange(lens.sum())
    sums = np.zeros(len(v))
    np.add.at(sums, np.repeat(np.arange(len(v)), lens), contrib[in_idx[idx]])
    if part_off is None:
        nv = np.full(len(v), float(n))
    else:
        po = np.asarray(part_off, np.int64)
        k = np.searchsorted(po, v, side="right") - 1
        nv = (po[k + 1] - po[k]).astype(np.float64)
    res = np.abs((1.0 - alpha) / nv + alpha * sums - R[v])
    return float(res.max()), float((res / R[v]).max()), int(len(v))


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_worklist
# launch from an ncu capture of the same workload, with the algorithmic bytes
# of that same launch (from the captured run's own counters), kept with a
# hash of the kernel's sources: a figure is reported only while the sources
# are unchanged. The work of an update varies from batch to batch (the
# asynchronous schedule), so a run reports the captured launch's DRAM bytes
# per algorithmic byte times its own algorithmic bytes per launch.
NOMINAL_HBM_GBS = 7900.0  # HBM3e bandwidth of the part, for context (the roofline uses the measured copy)

MEASURED_TRAFFIC = {
    # workload: (kernel source hash, DRAM bytes of the launch, its algorithmic bytes)
    ("rmat24-batch0.0001", "fp64", "worklist"): ("e43bc7b452f5cb31", 59.47e9, 55.94e9),
}


def kernel_source_hash():
    """Hash of the kernel's code (comments and blank lines left out, so that
    editing a comment does not retire a measurement)."""
    import re
    h = hashlib.sha256()
    for f in ("df.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2407_19562_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:16]


def measured_traffic(workload, precision, mode):
    """(DRAM bytes, algorithmic bytes) of the captured launch, or None."""
    rec = MEASURED_TRAFFIC.get((workload, precision, mode))
    if rec is None or rec[0] != kernel_source_hash() or rec[2] <= 0:
        return None
    return rec[1], rec[2]


def _random_gather_rate(torch, dev, elems, count, reps):
    """Best rate (gathers/s) of torch's index_select of `count` random int64
    from an array of `elems` int64, timed with CUDA events."""
    src = torch.zeros(elems, dtype=torch.int64, device=dev)
    idx = torch.randint(0, src.numel(), (count,), device=dev, dtype=torch.int64)
    out = torch.empty(count, dtype=torch.int64, device=dev)
    torch.index_select(src, 0, idx, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps):
        e0.record()
        torch.index_select(src, 0, idx, out=out)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del src, idx, out
    torch.cuda.empty_cache()
    return count / (best * 1e-3)


def random_line_ceiling(torch, dev, gib=4, count=1 << 26, reps=5, l2_mib=32):
    """Random-access ceilings of the memory system: 8-byte gathers at uniformly
    random positions (torch's index_select, CUDA events), once from a gib-GiB
    array (far larger than L2: every gather costs one DRAM line fetch, the
    device's ceiling for scattered lines) and once from an l2_mib-MiB array
    that L2 holds (the ceiling for scattered 32-byte sectors served by L2).
    The DF kernel's contribution and state reads meet these bounds long
    before the copy bandwidth."""
    rate = _random_gather_rate(torch, dev, gib << 27, count, reps)
    l2_rate = _random_gather_rate(torch, dev, l2_mib << 17, count, reps)
    return {"lines_per_s": rate, "gb_s_at_64B_lines": rate * 64 / 1e9,
            "how": f"index_select of {count} random int64 from a {gib} GiB array, best of {reps}",
            "l2_sectors_per_s": l2_rate,
            "l2_how": f"the same from a {l2_mib} MiB array (L2-resident)"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# --------------------------------------------------------------------------

def sample_spec(spec, cpu_scale: int):
    """The bounded sample of a workload the oracle is timed on: the same
    generator, edge factor and seed at R-MAT scale `cpu_scale`, or a grid of
    side 2^(cpu_scale / 2); and the ratio of the workload's edge draws to the
    sample's."""
    if spec["kind"] == "rmat":
        s = dict(spec, scale=min(cpu_scale, spec["scale"]))
        return s, float(2 ** (spec["scale"] - s["scale"]))
    L = min(1 << (cpu_scale // 2), spec["L"])
    return dict(spec, L=L), (spec["L"] / L) ** 2


def oracle_sample(spec, cpu_scale: int, batch_frac: float, steps: int, seed0: int = 100):
    """Times the oracle's apply + DF_LF (one core) on the bounded sample of a
    workload. Returns per-step ms of the sample, the factor that scales them
    to the workload, and a description. The batch is a fixed fraction of
    |E|, so the work of an update grows with |E|; the oracle's time per edge
    grows too as its arrays outgrow the CPU caches, so the scaled figure is a
    lower bound on the oracle's time at the workload's size."""
    import oracle
    sspec, factor = sample_spec(spec, cpu_scale)
    n, src, dst = make_graph(sspec)
    g = oracle.Graph.build(n, src, dst)
    R, _ = g.static_bb(tol=1e-13)  # R^0 converged to the frontier tolerance
    b = max(1, int(round(batch_frac * g.m)))
    times = []
    for i in range(steps):
        batch = make_batch(sspec, n, src, dst, b, seed0 + i)
        t0 = time.perf_counter()
        g, _ = g.apply(*batch)
        R, _ = g.df_lf(R)
        times.append((time.perf_counter() - t0) * 1e3)
    what = (f"R-MAT scale {sspec['scale']}, edge factor {sspec['edge_factor']}"
            if sspec["kind"] == "rmat" else f"grid {sspec['L']} x {sspec['L']}")
    desc = (f"oracle apply + DF_LF (Alg. 2, one thread) on {what} (n={n}, m={g.m}), batches of "
            f"{b} edges ({batch_frac:g}|E|, 80/20); ms/batch scaled by {factor:g}, the ratio of "
            f"the workload's edge draws to the sample's (a lower bound: the oracle's time per "
            f"edge grows with the graph)")
    return times, factor, desc


def cpu_baseline_entry(times, factor, desc, cores=1, growth=None):
    """The oracle's time per batch at the workload's size, from a bounded sample:
    scaled by the measured growth curve when one is given (growth =
    (value, growth per scale, smaller sample's ms)), else by the ratio of edge
    draws (a lower bound)."""
    sample_ms = statistics.mean(times)
    e = {"value": sample_ms * factor, "unit": UNIT, "cores": cores, "kind": "oracle",
         "sample": desc, "sample_ms_per_batch": sample_ms, "scale_factor": factor,
         "extrapolated": factor != 1.0, "linear_lower_bound": sample_ms * factor,
         "cpu": cpu_model(), "host_cpus": os.cpu_count()}
    if growth is not None:
        e["value"], e["growth_per_scale"], e["smaller_sample_ms_per_batch"] = growth
        e["scale_factor"] = e["value"] / sample_ms
        e["extrapolation"] = "measured growth curve: two samples two R-MAT scales apart"
    return e


def cpu_model():
    """Model name of the host CPU: lscpu's "Model name" (Arm hosts name the core
    there, e.g. Neoverse-V2), else /proc/cpuinfo's model name or part number."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def growth_extrapolation(spec, cpu_scale, batch_frac, sample_ms):
    """Extrapolates the oracle's ms per batch from the sample's scale to the
    workload's by a measured growth curve: one more sample two R-MAT scales
    below gives the growth per scale, g = (t(s) / t(s - 2))^(1/2), and the
    workload's time is t(s) * g^(S - s). Returns (value, g, the smaller
    sample's ms per batch) or None for non-R-MAT workloads."""
    if spec["kind"] != "rmat" or cpu_scale - 2 < 10 or spec["scale"] <= cpu_scale:
        return None
    small, _, _ = oracle_sample(spec, cpu_scale - 2, batch_frac, 2, seed0=140)
    t_small = statistics.mean(small)
    g = (sample_ms / t_small) ** 0.5 if t_small > 0 else 2.0
    return sample_ms * g ** (spec["scale"] - cpu_scale), g, t_small


# --------------------------------------------------------------------------
# arms
# --------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """Largest x over the ranks of the default process group (x itself when
    there is none or it has one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_batch(max_total_ms: float, steps: int, ws: int) -> float:
    """Whole-job ms per batch: every rank ran `steps` batches within the
    slowest rank's time."""
    return max_total_ms / (steps * ws)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the oracle baseline covers the single-graph workloads, not {args.workload}"}),
              flush=True)
        return
    spec = WORKLOADS[args.workload]
    times, factor, desc = oracle_sample(spec, args.cpu_scale, args.batch_frac,
                                        args.warmup + args.steps)
    growth = growth_extrapolation(spec, args.cpu_scale, args.batch_frac,
                                  statistics.mean(times[args.warmup:]))
    cpu = cpu_baseline_entry(times[args.warmup:], factor, desc, growth=growth)
    v = cpu["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}-batch{args.batch_frac:g}", "insert_frac": 0.8,
                   "precision": "fp64", "alpha": 0.85, "tol": 1e-10},
        "cpu_baseline": cpu,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import paper_2407_19562_gb300 as dfpr

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = WORKLOADS[args.workload]
    n, src, dst = make_graph(spec)
    cfg = dfpr.default_config(precision=dfpr.FP64 if args.precision == "fp64" else dfpr.FP32)
    stream = torch.cuda.Stream(device=dev)  # the library and the events share it
    torch.cuda.set_stream(stream)
    g = dfpr.graph_load(n, src, dst, cfg, stream=stream.cuda_stream)
    m0 = g.info()["m"]
    tol = 1e-10 if args.precision == "fp64" else 1e-7
    # R^0: static PageRank converged to the frontier tolerance (untimed), the
    # state a sequence of DF updates maintains
    st0 = dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, tol=tol / 1000.0,
                                                      max_iter=1000))
    if st0.status != dfpr.OK:
        raise RuntimeError(f"static pagerank did not converge: {st0.as_dict()}")
    b = max(1, int(round(args.batch_frac * m0)))
    mode = {"worklist": dfpr.WORKLIST, "round": dfpr.ROUND, "jacobi": dfpr.JACOBI}[args.mode]
    params = dfpr.default_params(mode=mode, tol=tol, timeout_ms=args.timeout_ms)
    total = args.warmup + args.steps
    batches = [make_batch(spec, n, src, dst, b, 100 + i + 1000 * rank) for i in range(total)]
    dev_batches = [[torch.from_numpy(x).to(dev) for x in bt] for bt in batches]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    for i in range(args.warmup):
        dfpr.apply_batch(g, *dev_batches[i])
        dfpr.df_pagerank(g, params)

    clocks = ClockSampler(torch.cuda.current_device())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = dfpr.kernel_launches()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0, e1 = ev[k]
        e0.record()
        dfpr.apply_batch(g, *dev_batches[args.warmup + k])
        st = dfpr.df_pagerank(g, params)
        e1.record()
        stats.append(st.as_dict())
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = dfpr.kernel_launches() - launches0 - 0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    my_total = sum(step_ms)
    my_total = max_over_ranks(my_total, dev)
    bad = [s for s in stats if s["status"] != dfpr.OK]

    # roofline of the persistent DF kernel (the dominant kernel)
    s_r = 8 if args.precision == "fp64" else 4
    kern_ms = [s["ms"] for s in stats]
    bytes_per = [algorithmic_bytes(s, s_r) for s in stats]
    achieved = sum(bytes_per) / (sum(kern_ms) * 1e-3) / 1e9 if sum(kern_ms) > 0 else 0.0
    peak, peak_kind = load_peaks()
    capture = measured_traffic(f"{args.workload}-batch{args.batch_frac:g}", args.precision, args.mode)
    # this run's DRAM bytes per launch, at the captured launch's bytes per algorithmic byte
    traffic = capture[0] / capture[1] * float(np.mean(bytes_per)) if capture else None
    ws_bytes, l2 = working_set_bytes(n, m0, s_r), l2_bytes(dev)
    ceiling = random_line_ceiling(torch, dev)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty(n, dtype=torch.float64, pin_memory=True)
        e2e_batches = [make_batch(spec, n, src, dst, b, 50_000 + i + 1000 * rank)
                       for i in range(args.steps)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for bt in e2e_batches:
            dfpr.apply_batch(g, *bt)
            dfpr.df_pagerank(g, params)
            dfpr.get_ranks(g, host_out)
        # whole job, like `value`: the slowest rank's time over all ranks' batches
        e2e_ms = job_ms_per_batch(max_over_ranks((time.perf_counter() - t0) * 1e3, dev),
                                  args.steps, ws)
        h2d = sum(x.nbytes for x in e2e_batches[0])
        e2e = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(8 * n)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        times, factor, desc = oracle_sample(spec, args.cpu_scale, args.batch_frac, 2)
        growth = growth_extrapolation(spec, args.cpu_scale, args.batch_frac, statistics.mean(times))
        cpu = cpu_baseline_entry(times, factor, desc, growth=growth)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    value = job_ms_per_batch(my_total, args.steps, ws)
    mean = lambda k: float(np.mean([s[k] for s in stats]))  # noqa: E731
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": my_total / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}-batch{args.batch_frac:g}", "n": n, "m": m0,
                   "batch_edges": b, "insert_frac": 0.8, "precision": args.precision,
                   "mode": args.mode, "alpha": 0.85, "tol": tol,
                   "accumulate": ("contributions as int64 round(C * 2^60), exact integer sums; "
                                  "ranks FP64" if args.precision == "fp64" else
                                  "FP32 contributions, TwoSum-compensated FP32 sums; FP64 "
                                  "dead-end sum, L-inf and normalisation"),
                   "l2": "flushed by a 256 MiB write between steps (outside the events)",
                   "replicas": ws},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "traffic_capture": ({"dram_bytes": capture[0], "algorithmic_bytes": capture[1],
                                          "ratio": capture[0] / capture[1],
                                          "how": "one ncu launch of this workload; traffic = "
                                                 "ratio x this run's algorithmic bytes"}
                                         if capture else None),
                     "peak_nominal": NOMINAL_HBM_GBS,
                     "kernel": "k_worklist (persistent DF kernel)",
                     "kernel_ms": float(np.mean(kern_ms)),
                     "algorithmic_bytes_per_launch": float(np.mean(bytes_per)),
                     # DRAM bytes of the ncu capture over this run's kernel time
                     "dram_achieved": (traffic / (float(np.mean(kern_ms)) * 1e-3) / 1e9
                                       if traffic else None),
                     "gteps": (float(np.mean([s["edges_gathered"] for s in stats]))
                               / (float(np.mean(kern_ms)) * 1e-3) / 1e9),
                     # a working set inside L2 never reaches HBM after the
                     # first touch: the HBM fraction is then low by design
                     "working_set_bytes": ws_bytes, "l2_bytes": l2,
                     "fits_l2": bool(l2) and ws_bytes <= l2,
                     # scattered 64-byte DRAM lines: the kernel's DRAM traffic
                     # in lines per second against the measured ceiling
                     "random_line_ceiling": ceiling,
                     "dram_lines_frac_of_ceiling": ((traffic / 64.0) / (float(np.mean(kern_ms)) * 1e-3)
                                                    / ceiling["lines_per_s"] if traffic else None)},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "work": {"processed": mean("processed"), "edges_gathered": mean("edges_gathered"),
                 "expansions": mean("expansions"), "edges_marked": mean("edges_marked"),
                 "pushes": mean("pushes"), "affected": mean("affected"),
                 "batches": mean("batches"), "tokens": mean("tokens"), "jobs": mean("jobs"),
                 "phase_share": phase_share(stats),
                 "apply_plus_df_ms_steps": step_ms, "algorithmic_bytes_steps": bytes_per,
                 "wall_s": t_wall,
                 "nonconverged_steps": len(bad)},
    }
    if ws == 1 and args.workload == "rmat24" and not args.no_extras:
        # the other configurations of the metric, each at its full size with
        # its own clocks and parity check (a failure is recorded, not fatal)
        g.free()
        del dev_batches, flush
        torch.cuda.empty_cache()
        extras = {}
        for key, fn in (("rmat24_fp32", lambda: extra_single(dfpr, torch, dev, "rmat24", "fp32")),
                        ("grid4096_fp32", lambda: extra_single(dfpr, torch, dev, "grid4096", "fp32")),
                        ("many256_fp32", lambda: extra_many(dfpr, torch, dev)),
                        ("serve8_fp64", lambda: extra_serve(dfpr, torch, dev))):
            t0 = time.perf_counter()
            try:
                extras[key] = fn()
            except Exception as e:  # noqa: BLE001 - recorded in the line
                extras[key] = {"error": f"{type(e).__name__}: {e}"}
            extras[key]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
        line["extras"] = extras
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------
# compact measurements of the other configurations, added to the default line
# --------------------------------------------------------------------------

def extra_single(dfpr, torch, dev, wname, precision, steps=5, warmup=3, batch_frac=1e-4):
    """One single-graph configuration at its full size: ms per batch (apply +
    update, CUDA events, L2 flushed between steps), the persistent kernel's
    algorithmic-byte rate, the work counters, clocks, and a parity check: Eq. 1
    residuals at sampled vertices, evaluated with numpy from the exported graph
    and ranks."""
    spec = WORKLOADS[wname]
    n, src, dst = make_graph(spec)
    prec = dfpr.FP64 if precision == "fp64" else dfpr.FP32
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    g = dfpr.graph_load(n, src, dst, dfpr.default_config(precision=prec), stream=stream.cuda_stream)
    m0 = g.info()["m"]
    tol = 1e-10 if precision == "fp64" else 1e-7
    dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, tol=tol / 1000.0, max_iter=1000))
    b = max(1, int(round(batch_frac * m0)))
    params = dfpr.default_params(tol=tol)
    batches = [[torch.from_numpy(x).to(dev) for x in make_batch(spec, n, src, dst, b, 300 + i)]
               for i in range(warmup + steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for i in range(warmup):
        dfpr.apply_batch(g, *batches[i])
        dfpr.df_pagerank(g, params)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms, stats = [], []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dfpr.apply_batch(g, *batches[warmup + k])
        st = dfpr.df_pagerank(g, params)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats.append(st.as_dict())
    clk = clocks.stop()
    s_r = 8 if precision == "fp64" else 4
    kern = float(np.mean([x["ms"] for x in stats]))
    byts = float(np.mean([algorithmic_bytes(x, s_r) for x in stats]))
    peak, peak_kind = load_peaks()
    R = dfpr.get_ranks(g)
    in_off, in_idx = dfpr.get_csc(g)
    res, res_rel, k = host_residual(R, in_off, in_idx)
    g.free()
    del flush
    torch.cuda.empty_cache()
    mean = lambda key: float(np.mean([x[key] for x in stats]))  # noqa: E731
    return {
        "workload": f"{wname}-batch{batch_frac:g}", "precision": precision, "n": n, "m": m0,
        "batch_edges": b, "ms_per_batch": float(np.mean(ms)), "kernel_ms": kern,
        "roofline": {"achieved": byts / (kern * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": byts / (kern * 1e-3) / 1e9 / peak, "peak_kind": peak_kind},
        "work": {"processed": mean("processed"), "edges_gathered": mean("edges_gathered"),
                 "expansions": mean("expansions"), "edges_marked": mean("edges_marked"),
                 "affected": mean("affected")},
        "nonconverged_steps": sum(x["status"] != dfpr.OK for x in stats),
        "parity": {"check": "Eq. 1 residual at sampled vertices (numpy, FP64, exported graph)",
                   "vertices": k, "max_abs": res, "max_rel": res_rel,
                   "bound": "tau = 1e-10 absolute" if precision == "fp64"
                   else "1e-6 relative"},
        "clocks": clk,
    }


def extra_many(dfpr, torch, dev, graphs=256, steps=2, warmup=1, precision="fp32"):
    """The many-graph configuration at N = 1: one persistent launch per step over
    all graphs against each graph updated alone in turn (per-graph latency from
    the step's start), with parity between the two forms and Eq. 1 residuals of
    the set's ranks."""
    a = argparse.Namespace(graphs=graphs, steps=steps, warmup=warmup, precision=precision,
                           autotune=True, timeout_ms=60000.0)
    return many_measure(a, quiet=True)


def extra_serve(dfpr, torch, dev, requests=150, load=0.8):
    """The serving configuration at one offered load (80 % of the measured
    single-stream capacity)."""
    a = argparse.Namespace(requests=requests, precision="fp64", timeout_ms=60000.0, units=2,
                           share_div=2)
    return serve_measure(a, loads=(load,), quiet=True)


def pct(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if len(xs) else None


def assign_by_edges(edges, ws):
    """Graphs of a set assigned to ws ranks: largest first, each to the rank
    with the fewest edges so far, since an update's work grows with the
    graph's edges. Returns one sorted list of graph indices per rank."""
    load = [0] * ws
    out = [[] for _ in range(ws)]
    for i in sorted(range(len(edges)), key=lambda i: (-edges[i], i)):
        r = min(range(ws), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += edges[i]
    return [sorted(x) for x in out]


def gather_to_rank0(xs):
    """Every rank's list, concatenated in rank order (xs itself without a
    process group). All ranks call it; only rank 0 needs the result."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(xs)
    got = [None] * dist.get_world_size()
    dist.all_gather_object(got, list(xs))
    return [x for part in got for x in part]


def many_measure(args, quiet=False):
    """Many graphs in one persistent launch per step (a set loaded with
    dfpr_graph_load_parts) against plain per-graph DF, one graph after another,
    on the same GPU. Per-graph latency of a step: from the step's start to the
    end of that graph's last recomputation."""
    import torch

    import paper_2407_19562_gb300 as dfpr
    ws, rank, local = dist_env()
    if ws > 1 and not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    elif ws == 1:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    specs = workloads.many_graph_specs(args.graphs, 1000)
    # the graphs shard across ranks with no collective on the data path
    mine = assign_by_edges([int(round(n * deg)) for n, deg, _ in specs], ws)[rank]
    graphs, off = [], [0]
    for i in mine:
        n, deg, frac = specs[i]
        n, src, dst = workloads.rmat_graph_n(n, deg, 1000 + i)
        graphs.append((n, src, dst, frac, i))
        off.append(off[-1] + n)
    off = np.array(off, np.int64)
    gsrc = np.concatenate([g[1] + o for g, o in zip(graphs, off)]).astype(np.int32)
    gdst = np.concatenate([g[2] + o for g, o in zip(graphs, off)]).astype(np.int32)
    prec = dfpr.FP64 if args.precision == "fp64" else dfpr.FP32
    tol = 1e-10 if args.precision == "fp64" else 1e-7
    cfg = dfpr.default_config(precision=prec)
    s_set = dfpr.graph_load_parts(off.astype(np.int32), gsrc, gdst, cfg, stream=stream.cuda_stream)
    st0 = dfpr.static_pagerank(s_set, dfpr.default_params(mode=dfpr.JACOBI, tol=tol / 1000, max_iter=1000))
    R0 = dfpr.get_ranks(s_set)
    # the set's update replays its device work from a CUDA graph (captured on
    # the first update, again only when a plan changes the launch)
    dfpr.set_capture(s_set, True)
    singles = []
    for i, (n, src, dst, frac, _) in enumerate(graphs):
        g = dfpr.graph_load(n, src, dst, cfg, stream=stream.cuda_stream)
        dfpr.set_ranks(g, np.ascontiguousarray(R0[off[i]:off[i + 1]]))
        singles.append(g)
    params = dfpr.default_params(tol=tol, timeout_ms=args.timeout_ms)
    params_alone = dfpr.default_params(tol=tol, timeout_ms=args.timeout_ms)
    tune_trials, tune_plans = [], []
    total = args.warmup + args.steps
    if args.autotune and args.warmup < 1:
        raise SystemExit("--autotune needs a warm-up step")

    def batches_for(step):
        out = []
        for n, src, dst, frac, gi in graphs:
            b = max(1, int(round(frac * len(src))))
            out.append(workloads.uniform_batch(n, b, 7000 + 1000 * step + gi, src, dst))
        return out

    set_lat, single_lat, set_step, single_step, set_kernel, set_bytes = [], [], [], [], [], []
    clocks = ClockSampler(torch.cuda.current_device())
    for step in range(total):
        if step == args.warmup:
            clocks.start()
        bl = batches_for(step)
        gb = [np.concatenate([b[k] + o for b, o in zip(bl, off)]).astype(np.int32) for k in range(4)]
        dev_gb = [torch.from_numpy(x).to(dev) for x in gb]
        dev_bl = [[torch.from_numpy(x).to(dev) for x in b] for b in bl]
        torch.cuda.synchronize()
        # the set: one apply + one persistent launch for every graph
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dfpr.apply_batch(s_set, *dev_gb)
        if args.autotune and step == 0:  # a warm-up step: tunes, then applies the update
            params, tune_plans, tune_trials, st = dfpr.autotune_plans(s_set, params)
        else:
            st = dfpr.df_pagerank(s_set, params)
        e1.record()
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1)
        part = dfpr.get_part_times(s_set)
        overhead = step_ms - st.ms
        lat = [overhead + t for t in part]
        # plain per-batch DF: each graph alone, one after another
        t_acc, lat1 = 0.0, []
        s0 = torch.cuda.Event(enable_timing=True)
        s0.record()
        evs = []
        for i, g in enumerate(singles):
            dfpr.apply_batch(g, *dev_bl[i])
            dfpr.df_pagerank(g, params_alone)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            evs.append(ev)
        torch.cuda.synchronize()
        lat1 = [s0.elapsed_time(ev) for ev in evs]
        if step >= args.warmup:
            set_lat += lat
            single_lat += lat1
            set_step.append(step_ms)
            single_step.append(lat1[-1])
            set_kernel.append(st.ms)
            set_bytes.append(algorithmic_bytes(st.as_dict(), 8 if prec == dfpr.FP64 else 4))
    clk = clocks.stop()
    cap_info = dfpr.capture_info(s_set)
    # both forms reach the same ranks (each graph's update is the same method)
    Rs = dfpr.get_ranks(s_set)
    in_off, in_idx = dfpr.get_csc(s_set)
    res, res_rel, nres = host_residual(Rs, in_off, in_idx, part_off=off)
    res_rel = max_over_ranks(res_rel, dev)
    diff = max(float(np.max(np.abs(Rs[off[i]:off[i + 1]] - dfpr.get_ranks(g))))
               for i, g in enumerate(singles))
    # whole job: every rank's graphs, timed by the slowest rank
    diff = max_over_ranks(diff, dev)
    set_total = max_over_ranks(float(np.sum(set_step)), dev)
    single_total = max_over_ranks(float(np.sum(single_step)), dev)
    kernel_total = max_over_ranks(float(np.sum(set_kernel)), dev)
    # roofline of the set's persistent kernel: algorithmic bytes of every
    # rank over the slowest rank's kernel time
    bytes_total = sum(gather_to_rank0([float(np.sum(set_bytes))]))
    peak, peak_kind = load_peaks()
    achieved = bytes_total / (kernel_total * 1e-3) / 1e9 if kernel_total > 0 else 0.0
    set_lat, single_lat = gather_to_rank0(set_lat), gather_to_rank0(single_lat)
    m_total = gather_to_rank0([int(len(gsrc))])
    s_set.free()
    for g in singles:
        g.free()
    torch.cuda.empty_cache()
    line = {
        "metric": "many-graph DF: ms/step and per-graph p50/p99 latency (batched vs per-graph)",
        "value": set_total / args.steps, "unit": "ms/step", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False, "scaling": "strong",
        "dtype": "f64" if prec == dfpr.FP64 else "f32",
        "data": "synthetic",
        "config": {"workload": f"many{args.graphs}: R-MAT n log-uniform [1e3,1e6], avg degree U[4,32], "
                               "batches 0.1-1% of each graph's edges (80/20)",
                   "graphs": args.graphs, "n_total": int(sum(n for n, _, _ in specs)),
                   "m_raw_total": int(sum(m_total)), "m_raw_per_rank": m_total,
                   "sharding": "graphs to ranks by greedy balance of edge draws, no collective",
                   "precision": args.precision},
        "batched": {"ms_per_step": set_total / args.steps, "kernel_ms": kernel_total / args.steps,
                    "update_from_cuda_graph": True, "captures_replays": list(cap_info),
                    "p50_ms": pct(set_lat, 50), "p99_ms": pct(set_lat, 99)},
        "per_graph_sequential": {"ms_per_step": single_total / args.steps,
                                 "p50_ms": pct(single_lat, 50), "p99_ms": pct(single_lat, 99)},
        "max_abs_diff_batched_vs_alone": diff,
        "parity": {"check": "Eq. 1 residual at sampled vertices of the set (numpy, FP64, "
                            "each graph's own n)", "vertices": nres, "max_rel": res_rel,
                   "bound": "1e-6 relative" if prec == dfpr.FP32 else "tau = 1e-10 absolute",
                   "batched_vs_alone": diff},
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "kernel": "k_worklist over the set (one launch per step)",
                     "algorithmic_bytes_per_launch": bytes_total / args.steps},
        "plan": {"mode": ["worklist", "round", "jacobi"][int(params.mode)],
                 "grid_ctas": int(params.grid_ctas), "gather_split": int(params.gather_split),
                 "mark_split": int(params.mark_split), "autotuned": bool(args.autotune),
                 "trials": ([{"plan": [int(x) for x in pl], "ms": float(t)}
                             for pl, t in zip(tune_plans, tune_trials)] if args.autotune else None)},
    }
    if not quiet and rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_many(args):
    many_measure(args)
    ws, _, _ = dist_env()
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()


def serve_measure(args, loads=(0.5, 0.8, 0.95), quiet=False):
    """Serving loop: 8 resident R-MAT graphs (scales 18,18,19,19,20,20,21,22,
    16 draws per vertex) receiving a Poisson stream of update batches, sizes
    log-uniform in [10, 1e5] (80/20), graph uniform. Three forms serve the same
    stream from the same starting ranks:
      continuous - dfpr_server over --units units (sets of graphs balanced by
                   edge draws, each with its own stream and worker): a
                   request is admitted as soon as its unit is idle and runs
                   beside the other units' updates;
      cycles     - dfpr_server over one set of the 8 graphs: every admitted
                   request of a cycle in one persistent launch, new requests
                   wait for the next cycle;
      plain      - dfpr_apply_batch + dfpr_df_pagerank per request, one at a
                   time in arrival order.
    Offered load: a fraction of the single-stream capacity (mean service time
    of requests served one at a time). Latency = completion - arrival (host
    monotonic clock)."""
    import threading as th

    import torch

    import paper_2407_19562_gb300 as dfpr
    ws, rank, local = dist_env()
    if ws > 1 and not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    elif ws == 1:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    scales = [18, 18, 19, 19, 20, 20, 21, 22]
    # the resident graphs shard across ranks; each rank serves the requests
    # to its own graphs, at the same fraction of its own measured capacity
    if ws > len(scales):
        raise SystemExit(f"serve8 shards {len(scales)} graphs: use at most {len(scales)} ranks")
    mine = assign_by_edges([16 << sc for sc in scales], ws)[rank]
    local_of = {gi: k for k, gi in enumerate(mine)}
    graphs, off = [], [0]
    for i in mine:
        n, src, dst = workloads.rmat_graph(scales[i], 16, 5000 + i)
        graphs.append((n, src, dst))
        off.append(off[-1] + n)
    off = np.array(off, np.int64)
    gsrc = np.concatenate([g[1] + o for g, o in zip(graphs, off)]).astype(np.int32)
    gdst = np.concatenate([g[2] + o for g, o in zip(graphs, off)]).astype(np.int32)
    prec = dfpr.FP64 if args.precision == "fp64" else dfpr.FP32
    tol = 1e-10 if args.precision == "fp64" else 1e-7
    cfg = dfpr.default_config(precision=prec)
    params = dfpr.default_params(tol=tol, timeout_ms=args.timeout_ms)
    # starting ranks: static PageRank of the set (untimed)
    gset = dfpr.graph_load_parts(off.astype(np.int32), gsrc, gdst, cfg, stream=None)
    dfpr.static_pagerank(gset, dfpr.default_params(mode=dfpr.JACOBI, tol=tol / 1000, max_iter=1000))
    R0 = dfpr.get_ranks(gset)
    gset.free()
    u = workloads.uniform01(6000, 1, 3 * 7 * args.requests * ws + 256 * ws)

    def make_requests(k0, count):
        """This rank's share of `count` requests of the global stream (graph
        uniform over all resident graphs), with graph ids local to the rank."""
        reqs = []
        for j in range(count):
            gi = int(u[k0 + 3 * j] * len(scales)) % len(scales)
            if gi not in local_of:
                continue
            b = int(round(10.0 ** (1.0 + 4.0 * u[k0 + 3 * j + 1])))
            n, src, dst = graphs[local_of[gi]]
            reqs.append((local_of[gi], workloads.uniform_batch(n, b, 60000 + k0 + j, src, dst)))
        return reqs

    def load_groups(k):
        """The rank's graphs in k units (sets of graphs balanced by edge draws;
        a unit of one graph is loaded alone). Returns the units, each graph's
        part index in the server's numbering (units in order), and each
        graph's (unit, vertex offset in the unit)."""
        k = max(1, min(k, len(graphs)))
        groups = assign_by_edges([len(g[1]) for g in graphs], k)
        units, part_of, where = [], [0] * len(graphs), [None] * len(graphs)
        base = 0
        for grp in groups:
            if len(grp) == 1:
                i = grp[0]
                n, src, dst = graphs[i]
                h = dfpr.graph_load(n, src, dst, cfg, stream=None)
                dfpr.set_ranks(h, np.ascontiguousarray(R0[off[i]:off[i + 1]]))
                part_of[i], where[i] = base, (len(units), 0)
            else:
                o = np.cumsum([0] + [graphs[i][0] for i in grp])
                us = np.concatenate([graphs[i][1] + o[j] for j, i in enumerate(grp)]).astype(np.int32)
                ud = np.concatenate([graphs[i][2] + o[j] for j, i in enumerate(grp)]).astype(np.int32)
                h = dfpr.graph_load_parts(o.astype(np.int32), us, ud, cfg, stream=None)
                dfpr.set_ranks(h, np.concatenate([R0[off[i]:off[i + 1]] for i in grp]))
                for j, i in enumerate(grp):
                    part_of[i], where[i] = base + j, (len(units), int(o[j]))
            units.append(h)
            base += len(grp)
        return units, part_of, where

    def final_ranks(units, where):
        Rs = [dfpr.get_ranks(h) for h in units]
        return [Rs[u][o:o + graphs[i][0]].copy() for i, (u, o) in enumerate(where)]

    def run_form(form, reqs, gaps):
        k = {"cycles": 1, "plain": len(graphs)}.get(form, getattr(args, "units", 2))
        held, part_of, where = load_groups(k)
        lat, edges = [], sum(len(b[0]) + len(b[2]) for _, b in reqs)
        t0 = time.perf_counter()
        if form == "plain":
            t = t0
            done = []
            for j, (gi, batch) in enumerate(reqs):
                t += gaps[j]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                dfpr.apply_batch(held[where[gi][0]], *batch)
                st = dfpr.df_pagerank(held[where[gi][0]], params)
                done.append((t, time.perf_counter(), st.status))
            lat = [(b - a) * 1e3 for a, b, _ in done]
            span = done[-1][1] - t0
            bad = sum(x[2] != dfpr.OK for x in done)
            updates = len(reqs)
        else:
            # continuous: every launch capped at a share of a wave (half by
            # default), so that units' updates run side by side
            share = (5 * torch.cuda.get_device_properties(dev).multi_processor_count) // \
                max(1, getattr(args, "share_div", 2))
            srv = dfpr.server_create(held, params, max_slots=64, mem_fraction=0.5,
                                     grid_share=share if form == "continuous" else 0)
            ids = [None] * len(reqs)

            def submitter():
                t = t0
                for j, (gi, batch) in enumerate(reqs):
                    t += gaps[j]
                    d = t - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    ids[j] = srv.submit(part_of[gi], *batch)

            thr = th.Thread(target=submitter)
            thr.start()
            thr.join()
            infos = [srv.wait(r) for r in ids]
            srv.destroy()
            lat = [i.done_ms - i.submit_ms for i in infos]
            span = (max(i.done_ms for i in infos) - min(i.submit_ms for i in infos)) / 1e3
            bad = sum(i.status != dfpr.OK for i in infos)
            updates = len({i.cycle for i in infos})
        R = final_ranks(held, where)
        for h in held:
            h.free()
        lat = gather_to_rank0(lat)
        tot = gather_to_rank0([(edges, len(reqs), span, updates, bad)])
        return R, {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(np.mean(lat)),
                   "updates_per_s": sum(t[0] / t[2] for t in tot if t[2] > 0),
                   "requests_per_s": sum(t[1] / t[2] for t in tot if t[2] > 0),
                   "launches": sum(t[3] for t in tot), "bad": sum(t[4] for t in tot)}

    # single-stream capacity: requests served one at a time, back to back
    cal = make_requests(0, 40 * ws)
    units, _, where = load_groups(len(graphs))
    svc = []
    for gi, batch in cal:
        t = time.perf_counter()
        dfpr.apply_batch(units[where[gi][0]], *batch)
        dfpr.df_pagerank(units[where[gi][0]], params)
        svc.append((time.perf_counter() - t) * 1e3)
    for h in units:
        h.free()
    mean_svc = float(np.mean(svc))
    svc_all = gather_to_rank0([mean_svc])
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    points = []
    k = max(200, 120 * ws + 8)  # past the calibration draws
    for load in loads:
        reqs = make_requests(k, args.requests * ws)
        k += 3 * args.requests * ws
        if not reqs:
            raise SystemExit("a rank drew no requests: raise --requests")
        rate = load / (mean_svc / 1e3)
        rng = np.random.default_rng(int(load * 100) + 1000 * rank)
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        out, ranks = {"load": load, "offered_req_per_s": rate}, {}
        for form in ("continuous", "cycles", "plain"):
            ranks[form], out[form] = run_form(form, reqs, gaps)
        # every form applied the same requests in the same order per graph
        diff = max(float(np.max(np.abs(a - b))) for f in ("continuous", "cycles")
                   for a, b in zip(ranks[f], ranks["plain"]))
        out["max_abs_diff_vs_plain"] = max_over_ranks(diff)
        points.append(out)
    clk = clocks.stop()
    line = {
        "metric": "serving: per-batch p50/p99 latency (ms) and updates/s; continuous units vs "
                  "cycles vs plain per-batch calls",
        "value": points[-1]["continuous"]["p99_ms"],
        "unit": f"ms (p99 at {int(round(100 * loads[-1]))}% load, continuous)",
        "n_gpus": ws, "higher_is_better": False, "scaling": "weak",
        "dtype": "f64" if prec == dfpr.FP64 else "f32", "data": "synthetic",
        "config": {"workload": "serve8: R-MAT scales 18,18,19,19,20,20,21,22; Poisson arrivals; "
                               "batch sizes log-uniform [10,1e5], 80/20",
                   "requests_per_point": args.requests, "mean_service_ms": svc_all,
                   "continuous_grid_share": f"1/{max(1, getattr(args, 'share_div', 2))} of a wave",
                   "continuous_units": getattr(args, "units", 2),
                   "sharding": "graphs to ranks by greedy balance of edge draws; each rank "
                               "at the load fraction of its own capacity",
                   "precision": args.precision},
        "points": points,
        "parity": {"check": "final ranks of every graph, continuous and cycles against plain "
                            "per-batch updates of the same requests",
                   "bound": 1e-9 if prec == dfpr.FP64 else "1e-6 relative"},
        "clocks": clk,
    }
    if not quiet and rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_serve(args):
    serve_measure(args)
    ws, _, _ = dist_env()
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()


def run_faults(args):
    """Thread delays and crash-stops (Sec. 5.3, 5.4) on the GPU: one DF update
    of R-MAT scale 20 at batch 1e-4 |E| under each fault setting, for the
    barrier-based jacobi schedule (DF_BB), the round schedule (DF_LF, Alg. 2)
    and the worklist schedule. A warp stands for a thread; a delay is a
    bounded sleep after a batch of vertices, with the given probability per
    vertex; a crash-stop warp returns at a random batch boundary. Error = L-inf
    against the fault-free result of the same schedule."""
    import torch

    import paper_2407_19562_gb300 as dfpr
    torch.cuda.set_device(0)
    n, src, dst = workloads.rmat_graph(20, 16, 3)
    tol = 1e-10
    g = dfpr.graph_load(n, src, dst, stream=None)
    dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, tol=tol / 1000, max_iter=1000))
    R0 = dfpr.get_ranks(g)
    m0 = g.info()["m"]
    b = max(1, int(round(args.batch_frac * m0)))
    batch = workloads.uniform_batch(n, b, 100, src, dst)
    grid = 64  # CTAs: 512 warps stand for the threads

    def one(mode, **kw):
        h = dfpr.graph_load(n, src, dst, stream=None)
        dfpr.set_ranks(h, R0)
        dfpr.apply_batch(h, *batch)
        p = dfpr.default_params(mode=getattr(dfpr, mode), grid_ctas=grid, timeout_ms=args.timeout_ms, **kw)
        try:
            st = dfpr.df_pagerank(h, p)
        except dfpr.DfprError as e:
            return {"status": int(e.status), "note": str(e)}, None
        return {"status": int(st.status), "ms": st.ms, "processed": int(st.processed),
                "passes": int(st.passes)}, dfpr.get_ranks(h)

    base = {}
    rows = []
    for mode in ("JACOBI", "ROUND", "WORKLIST"):
        r, R = one(mode)
        base[mode] = R
        rows.append({"mode": mode, "fault": "none", **r, "err": 0.0})
    for mode in ("JACOBI", "ROUND", "WORKLIST"):
        for prob in (1e-5, 1e-4):
            for us in (200.0, 1000.0):
                r, R = one(mode, fault_delay_prob=prob, fault_delay_us=us, fault_seed=1)
                err = float(np.max(np.abs(R - base[mode]))) if R is not None else None
                rows.append({"mode": mode, "fault": f"delay p={prob:g}/vertex {us:g}us", **r, "err": err})
        for crashed in (1, 64, 256, 448):
            r, R = one(mode, fault_crash_warps=crashed, fault_seed=1)
            err = float(np.max(np.abs(R - base[mode]))) if R is not None and r["status"] == 0 else None
            rows.append({"mode": mode, "fault": f"crash {crashed}/512 warps", **r, "err": err})
    line = {"metric": "DF update ms/batch under simulated thread delays and crash-stops",
            "unit": "ms/batch", "n_gpus": 1, "higher_is_better": False, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"rmat20-batch{args.batch_frac:g}", "n": n, "m": m0,
                       "batch_edges": b, "warps": grid * 8, "timeout_ms": args.timeout_ms},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """DF against ND and Static across batch sizes (the comparison of Sec.
    5.2.2) on one graph: for each size 10^k |E|, k = -7 .. -1, a sequence of
    batches; each is applied (timed) and updated by DF (timed); then the
    previous ranks are restored and ND is timed, and Static from 1/n. The
    sequence continues from DF's ranks. Times by CUDA events on the library's
    stream; L2 flushed before every timed call."""
    import torch

    import paper_2407_19562_gb300 as dfpr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spec = WORKLOADS["rmat24" if args.graph == "rmat24" else args.graph]
    n, src, dst = make_graph(spec)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    g = dfpr.graph_load(n, src, dst, stream=stream.cuda_stream)
    m0 = g.info()["m"]
    tol = 1e-10
    dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, tol=tol / 1000, max_iter=1000))
    params = dfpr.default_params(tol=tol, timeout_ms=args.timeout_ms)
    pjac = dfpr.default_params(tol=tol, mode=dfpr.JACOBI, timeout_ms=args.timeout_ms)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    rows = []
    reps = max(1, args.steps)
    for k in range(-7, 0):
        b = max(1, int(round(10.0 ** k * m0)))
        acc = {"apply": [], "df": [], "nd": [], "static": [], "nd_bb": [], "static_bb": []}
        bad = 0
        for i in range(reps):
            batch = [torch.from_numpy(x).to(dev) for x in
                     make_batch(spec, n, src, dst, b, 5000 + 100 * (k + 8) + i)]
            torch.cuda.synchronize()
            R_prev = dfpr.get_ranks(g)
            t_apply, _ = timed(lambda: dfpr.apply_batch(g, *batch))
            t_df, st = timed(lambda: dfpr.df_pagerank(g, params))
            bad += st.status != dfpr.OK
            R_df = dfpr.get_ranks(g)
            dfpr.set_ranks(g, R_prev)
            t_nd, st2 = timed(lambda: dfpr.nd_pagerank(g, params))
            bad += st2.status != dfpr.OK
            t_st, st3 = timed(lambda: dfpr.static_pagerank(g, params))
            bad += st3.status != dfpr.OK
            # the paper's barrier-based forms: every vertex, every iteration
            dfpr.set_ranks(g, R_prev)
            t_ndbb, st4 = timed(lambda: dfpr.nd_pagerank(g, pjac))
            t_stbb, st5 = timed(lambda: dfpr.static_pagerank(g, pjac))
            bad += (st4.status != dfpr.OK) + (st5.status != dfpr.OK)
            dfpr.set_ranks(g, R_df)
            for key, t in (("apply", t_apply), ("df", t_df), ("nd", t_nd), ("static", t_st),
                           ("nd_bb", t_ndbb), ("static_bb", t_stbb)):
                acc[key].append(t)
        med = {key: float(np.median(v)) for key, v in acc.items()}
        rows.append({"batch_frac": 10.0 ** k, "batch_edges": b, "ms_apply": med["apply"],
                     "ms_df": med["df"], "ms_nd": med["nd"], "ms_static": med["static"],
                     "ms_nd_bb": med["nd_bb"], "ms_static_bb": med["static_bb"],
                     "df_vs_nd": (med["nd"]) / (med["apply"] + med["df"]),
                     "df_vs_static": (med["static"]) / (med["apply"] + med["df"]),
                     "df_vs_nd_bb": med["nd_bb"] / (med["apply"] + med["df"]),
                     "df_vs_static_bb": med["static_bb"] / (med["apply"] + med["df"]),
                     "not_ok": bad})
    line = {"metric": "DF vs ND vs Static ms per batch across batch sizes", "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.graph} batches 1e-7..1e-1 |E| (80/20)", "n": n, "m": m0,
                       "repeats": reps, "mode": "worklist (DF, ND, Static); jacobi (ND_BB, Static_BB)",
                       "note": "df_vs_* = that method's update time / (apply + DF) time"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_stream(args):
    """Insert-only updates in edge order (the protocol of Sec. 5.1.4 for the
    temporal graphs): the first 90% of an R-MAT edge stream (scale 24, 16
    draws per vertex, drawing order standing in for time) is loaded, then the
    following edges arrive in batches of 1e-4 and 1e-3 of the stream. Each
    batch: apply + DF timed; previous ranks restored, ND timed; Static timed."""
    import torch

    import paper_2407_19562_gb300 as dfpr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n, src, dst = workloads.rmat_graph(24, 16, 3)
    ET = len(src)
    pre = int(0.9 * ET)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    g = dfpr.graph_load(n, src[:pre], dst[:pre], stream=stream.cuda_stream)
    dfpr.static_pagerank(g, dfpr.default_params(mode=dfpr.JACOBI, tol=1e-13, max_iter=1000))
    params = dfpr.default_params(tol=1e-10, timeout_ms=args.timeout_ms)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    empty = torch.zeros(0, dtype=torch.int32, device=dev)

    def timed(fn):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    rows = []
    pos = pre
    for frac in (1e-4, 1e-3):
        b = int(round(frac * ET))
        acc = {"apply": [], "df": [], "nd": [], "static": []}
        real = []
        bad = 0
        for i in range(max(1, args.steps)):
            s_ = torch.from_numpy(np.ascontiguousarray(src[pos:pos + b])).to(dev)
            d_ = torch.from_numpy(np.ascontiguousarray(dst[pos:pos + b])).to(dev)
            pos += b
            torch.cuda.synchronize()
            R_prev = dfpr.get_ranks(g)
            t_apply, nreal = timed(lambda: dfpr.apply_batch(g, empty, empty, s_, d_))
            real.append(int(nreal[1]))
            t_df, st = timed(lambda: dfpr.df_pagerank(g, params))
            R_df = dfpr.get_ranks(g)
            dfpr.set_ranks(g, R_prev)
            t_nd, st2 = timed(lambda: dfpr.nd_pagerank(g, params))
            t_st, st3 = timed(lambda: dfpr.static_pagerank(g, params))
            bad += sum(x.status != dfpr.OK for x in (st, st2, st3))
            dfpr.set_ranks(g, R_df)
            for key, t in (("apply", t_apply), ("df", t_df), ("nd", t_nd), ("static", t_st)):
                acc[key].append(t)
        med = {key: float(np.median(v)) for key, v in acc.items()}
        rows.append({"batch_frac_of_stream": frac, "batch_edges": b,
                     "new_edges_median": int(np.median(real)), "ms_apply": med["apply"],
                     "ms_df": med["df"], "ms_nd": med["nd"], "ms_static": med["static"],
                     "df_vs_nd": med["nd"] / (med["apply"] + med["df"]),
                     "df_vs_static": med["static"] / (med["apply"] + med["df"]), "not_ok": bad})
    line = {"metric": "insert-only stream: DF vs ND vs Static ms per batch", "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "R-MAT scale 24 edge stream, 90% preloaded, insert-only batches",
                       "n": n, "stream_edges": ET, "repeats": max(1, args.steps), "mode": "worklist"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "many256":
        run_many(args)
    elif args.workload == "serve8":
        run_serve(args)
    elif args.workload == "faults":
        run_faults(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "stream":
        run_stream(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
