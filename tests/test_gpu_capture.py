"""CUDA-graph replay of the DF update (dfpr_graph_set_capture) on a set of
graphs, the many-graph step: a sequence of batches of different sizes is
applied to two copies of the same set, one updated eagerly and one from the
captured graph; after every batch both equal each other and the oracle's
reference ranks of every graph, and the captured copy replays one graph for
batches of any size."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9
SPECS = [(3000, 8.0), (700, 5.0), (20000, 12.0), (9000, 6.0)]


def test_replay_equals_eager_equals_oracle(gpu_lib):
    dfpr = gpu_lib
    graphs, off = [], [0]
    for i, (n, deg) in enumerate(SPECS):
        n, src, dst = workloads.rmat_graph_n(n, deg, 2100 + i)
        og = oracle.Graph.build(n, src, dst)
        graphs.append(dict(n=n, src=src, dst=dst, og=og, ref=og.reference()[0]))
        off.append(off[-1] + n)
    off = np.array(off, np.int32)
    gsrc = np.concatenate([g["src"] + o for g, o in zip(graphs, off)]).astype(np.int32)
    gdst = np.concatenate([g["dst"] + o for g, o in zip(graphs, off)]).astype(np.int32)
    R0 = np.concatenate([g["ref"] for g in graphs])
    eager = dfpr.graph_load_parts(off, gsrc, gdst, stream=None)
    replay = dfpr.graph_load_parts(off, gsrc, gdst, stream=None)
    for h in (eager, replay):
        h.set_ranks(R0)
    replay.set_capture(True)
    for step, b in enumerate((40, 400, 7, 120)):
        bl = [workloads.uniform_batch(g["n"], b, 2200 + 10 * step + i, g["src"], g["dst"])
              for i, g in enumerate(graphs)]
        batch = [np.concatenate([x[k] + o for x, o in zip(bl, off)]).astype(np.int32) for k in range(4)]
        for h in (eager, replay):
            h.apply_batch(*batch)
        st_e = eager.df_pagerank()
        st_r = replay.df_pagerank()
        assert st_e.status == dfpr.OK and st_r.status == dfpr.OK
        assert st_r.processed > 0 and st_r.ms > 0
        Re, Rr = eager.get_ranks(), replay.get_ranks()
        assert float(np.max(np.abs(Re - Rr))) <= LINF64
        for i, g in enumerate(graphs):
            g["og"], _ = g["og"].apply(*bl[i])
            ref, _ = g["og"].reference()
            assert float(np.max(np.abs(Rr[off[i]:off[i + 1]] - ref))) <= LINF64, (step, i)
        assert np.array_equal(eager.get_csr()[1], replay.get_csr()[1])
    captures, replays = replay.capture_info()
    assert replays == 4 and 1 <= captures < replays     # batches of other sizes replay it
    assert eager.capture_info() == (0, 0)
    replay.set_capture(False)
    for h in (eager, replay):
        h.free()
