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


def test_units_update_continuously_and_match_oracle(gpu_lib, served):
    # every graph its own unit (own stream, own worker): requests are admitted
    # whenever their graph is idle, not at cycle boundaries, and the results
    # are those of the set served in cycles and of the oracle
    graphs, off, _, _, reqs = served
    units = []
    for g in graphs:
        h = gpu_lib.graph_load(g["n"], g["src"], g["dst"], stream=None)
        h.set_ranks(g["ref0"])
        units.append(h)
    sms = __import__("torch").cuda.get_device_properties(0).multi_processor_count
    srv = gpu_lib.server_create(units, max_slots=64, grid_share=2 * sms)
    ids = [srv.submit(i, *batch) for i, batch in reqs]
    infos = [srv.wait(r) for r in ids]
    srv.destroy()
    assert all(i.status == gpu_lib.OK for i in infos)
    for i in infos:
        assert i.submit_ms <= i.admit_ms <= i.done_ms
    # updates of different units overlapped in time
    spans = sorted({(i.cycle, i.admit_ms, i.done_ms) for i in infos}, key=lambda t: t[1])
    assert any(b[1] < a[2] for a, b in zip(spans, spans[1:]))
    R_mix, _ = serve_all(gpu_lib, served, max_slots=64)
    for k, g in enumerate(graphs):
        R = units[k].get_ranks()
        assert np.max(np.abs(R - g["ref1"])) <= LINF64, k
        assert np.max(np.abs(R - R_mix[off[k]:off[k + 1]])) <= LINF64, k


def test_request_for_an_idle_unit_is_admitted_during_another_update(gpu_lib):
    import time
    big_n, big_s, big_d = workloads.rmat_graph(17, 16, 41)
    small_n, small_s, small_d = workloads.rmat_graph_n(3000, 8.0, 42)
    o_big = oracle.Graph.build(big_n, big_s, big_d)
    o_small = oracle.Graph.build(small_n, small_s, small_d)
    R_big, _ = o_big.reference()
    R_small, _ = o_small.reference()
    big_batch = workloads.uniform_batch(big_n, 60000, 43, big_s, big_d)
    small_batch = workloads.uniform_batch(small_n, 50, 44, small_s, small_d)
    ref_big, _ = o_big.apply(*big_batch)[0].reference()
    ref_small, _ = o_small.apply(*small_batch)[0].reference()
    a = gpu_lib.graph_load(big_n, big_s, big_d, stream=None)
    b = gpu_lib.graph_load(small_n, small_s, small_d, stream=None)
    a.set_ranks(R_big)
    b.set_ranks(R_small)
    sms = __import__("torch").cuda.get_device_properties(0).multi_processor_count
    srv = gpu_lib.server_create([a, b], max_slots=8, grid_share=2 * sms)
    ra = srv.submit(0, *big_batch)
    # wait until the big update is running, then submit for the idle unit
    t0 = time.perf_counter()
    time.sleep(0.002)
    rb = srv.submit(1, *small_batch)
    ib, ia = srv.wait(rb), srv.wait(ra)
    srv.destroy()
    assert ia.status == gpu_lib.OK and ib.status == gpu_lib.OK
    assert ib.submit_ms < ia.done_ms, "the small request arrived after the big update ended"
    assert ib.admit_ms < ia.done_ms          # admitted while the other update ran
    assert ib.cycle != ia.cycle
    assert np.max(np.abs(a.get_ranks() - ref_big)) <= LINF64
    assert np.max(np.abs(b.get_ranks() - ref_small)) <= LINF64
    assert time.perf_counter() - t0 < 60
