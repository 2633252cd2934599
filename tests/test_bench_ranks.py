"""The multi-rank path of bench.py on the CPU: two gloo ranks, 127.0.0.1
rendezvous. The timing aggregate is the slowest rank's total, under torchrun
the reference arm prints one line, from rank 0 only, and a graph set shards
over ranks by edges, with per-graph results gathered on rank 0."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    bench = load_bench()
    total = [120.0, 150.0][rank]          # per-rank sum of step times (ms)
    m = bench.max_over_ranks(total)
    out[rank] = (m, bench.job_ms_per_batch(m, 10, 2))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    port = free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(port, out), nprocs=2, join=True)
        got = dict(out)
    assert got[0] == got[1] == (150.0, 7.5)  # 2 ranks x 10 batches within 150 ms


def test_single_process_aggregate_is_identity():
    bench = load_bench()
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_ms_per_batch(100.0, 10, 1) == 10.0


def test_reference_arm_prints_once_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--cpu-scale", "10"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_graph_set_assignment_covers_and_balances():
    bench = load_bench()
    rng = np.random.default_rng(3)
    edges = [int(x) for x in rng.integers(1_000, 1_000_000, 256)]
    for ws in (1, 2, 3, 8):
        parts = bench.assign_by_edges(edges, ws)
        assert len(parts) == ws
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(edges)))          # each graph exactly once
        loads = [sum(edges[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(edges)    # greedy, largest first
        assert bench.assign_by_edges(edges, ws) == parts  # deterministic
    assert bench.assign_by_edges([5, 3], 4) == [[0], [1], [], []]


def _gather_main(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    bench = load_bench()
    mine = [[1.5, 2.5], [7.0]][rank]                 # per-graph latencies of this rank
    out[rank] = bench.gather_to_rank0(mine)
    dist.destroy_process_group()


def test_per_graph_results_gathered_over_two_gloo_ranks():
    port = free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_gather_main, args=(port, out), nprocs=2, join=True)
        got = dict(out)
    assert got[0] == [1.5, 2.5, 7.0]
    bench = load_bench()
    assert bench.gather_to_rank0([4.0]) == [4.0]        # no process group: itself
