"""The serving runtime (dfpr_server_*): requests served together in one cycle
give the same ranks as the same requests served one per cycle, and both match
the oracle's reference for each graph after its requests."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

LINF64 = 1e-9
SPECS = [(2000, 8.0), (9000, 12.0), (500, 5.0), (30000, 10.0)]


@pytest.fixture(scope="module")
def served():
    graphs, off = [], [0]
    for i, (n, deg) in enumerate(SPECS):
        n, src, dst = workloads.rmat_graph_n(n, deg, 800 + i)
        g0 = oracle.Graph.build(n, src, dst)
        ref0, _ = g0.reference()
        graphs.append(dict(n=n, src=src, dst=dst, g=g0, ref0=ref0))
        off.append(off[-1] + n)
    # 3 requests per graph, sizes 10 .. 2000, interleaved by graph
    reqs = []
    for k in range(3):
        for i, g in enumerate(graphs):
            b = [10, 300, 2000][(k + i) % 3]
            reqs.append((i, workloads.uniform_batch(g["n"], b, 900 + 10 * k + i, g["src"], g["dst"])))
    for i, g in enumerate(graphs):
        og = g["g"]
        for j, batch in reqs:
            if j == i:
                og, _ = og.apply(*batch)
        g["ref1"], _ = og.reference()
    gsrc = np.concatenate([g["src"] + o for g, o in zip(graphs, off)]).astype(np.int32)
    gdst = np.concatenate([g["dst"] + o for g, o in zip(graphs, off)]).astype(np.int32)
    return graphs, np.array(off, np.int32), gsrc, gdst, reqs


def serve_all(gpu_lib, served, max_slots):
    graphs, off, gsrc, gdst, reqs = served
    s = gpu_lib.graph_load_parts(off, gsrc, gdst)
    s.set_ranks(np.concatenate([g["ref0"] for g in graphs]))
    srv = gpu_lib.server_create(s, max_slots=max_slots)
    ids = [srv.submit(i, *batch) for i, batch in reqs]
    with pytest.raises(gpu_lib.DfprError) as e:  # the graph belongs to the server
        s.get_ranks()
    assert e.value.status == gpu_lib.EBUSY
    infos = [srv.wait(r) for r in ids]
    srv.destroy()
    return s.get_ranks(), infos


def test_mix_equals_alone_equals_oracle(gpu_lib, served):
    graphs, off = served[0], served[1]
    R_mix, info_mix = serve_all(gpu_lib, served, max_slots=64)
    R_one, info_one = serve_all(gpu_lib, served, max_slots=1)
    assert all(i.status == gpu_lib.OK for i in info_mix + info_one)
    assert all(i.cycle_requests == 1 for i in info_one)
    assert len({i.cycle for i in info_one}) == len(info_one)
    assert any(i.cycle_requests > 1 for i in info_mix)   # requests shared cycles
    for i in info_mix + info_one:
        assert i.submit_ms <= i.admit_ms <= i.done_ms
    for k, g in enumerate(graphs):
        a, b = off[k], off[k + 1]
        assert np.max(np.abs(R_mix[a:b] - g["ref1"])) <= LINF64, k
        assert np.max(np.abs(R_one[a:b] - g["ref1"])) <= LINF64, k
        assert np.max(np.abs(R_mix[a:b] - R_one[a:b])) <= LINF64, k


def test_server_rejects_bad_requests(gpu_lib, served):
    graphs, off, gsrc, gdst, _ = served
    s = gpu_lib.graph_load_parts(off, gsrc, gdst)
    srv = gpu_lib.server_create(s, max_slots=4)
    bad = np.array([graphs[0]["n"]], np.int32)  # outside graph 0
    with pytest.raises(gpu_lib.DfprError):
        srv.submit(0, bad, bad, bad[:0], bad[:0])
    with pytest.raises(gpu_lib.DfprError):
        srv.submit(len(graphs), bad[:0], bad[:0], bad[:0], bad[:0])
    rid = srv.submit(1, np.zeros(0, np.int32), np.zeros(0, np.int32),
                     np.array([0], np.int32), np.array([1], np.int32))
    assert srv.wait(rid).status == gpu_lib.OK
    srv.drain()
    srv.destroy()
    s.get_ranks()  # usable again once the server is gone
