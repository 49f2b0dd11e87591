"""Serving with continuous batching: every answer is the same alone and in the mix (integers,
compared exactly), requests submitted while a launch runs join it, and admission under a tiny
memory budget queues requests instead of failing them."""
import time

import numpy as np
import pytest

import oracle
from paper_2204_10402_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vc():
    import torch
    assert torch.cuda.is_available()
    import paper_2204_10402_gb300 as vc
    from paper_2204_10402_gb300 import build
    build.build()
    vc.load()
    return vc


def mixed_requests(count, seed0):
    """(graph, kind, k, expected answer) with answers from the CPU oracle."""
    out = []
    for i in range(count):
        u = G.uniform01(seed0 + i, 4)
        if u[0] < 0.5:
            n = 20 + int(u[1] * 70)
            g = G.gnp(n, 0.05 + 0.15 * u[2], seed0 + i, draw_offset=4)
        else:
            n = 100 + int(u[1] * 900)
            g = G.chung_lu(n, 4.0 + 2.5 * u[2], seed0 + i)
        best, _, _ = oracle.mvc(g)
        if u[3] < 0.3:
            out.append((g, 0, 0, best))
        else:
            k = best - (1 if u[3] < 0.65 else 0)
            out.append((g, 1, k, int(k >= best)))
    return out


def run_alone(vc, reqs):
    got = []
    for g, kind, k, _ in reqs:
        if kind == 0:
            got.append(vc.mvc(g.offsets, g.neighbors, want_cover=False).value)
        else:
            got.append(vc.pvc(g.offsets, g.neighbors, k, want_cover=False).value)
    return got


@pytest.mark.parametrize("bit_rows", [0, 1])
def test_mix_equals_alone_and_oracle(vc, bit_rows):
    reqs = mixed_requests(80, 120000)
    alone = run_alone(vc, reqs)
    assert alone == [r[3] for r in reqs]
    with vc.Server(max_n=1000, config=vc.make_config(bit_rows=bit_rows)) as srv:
        ids = [srv.submit(g.offsets, g.neighbors, kind, k) for g, kind, k, _ in reqs]
        srv.drain(timeout_ms=120000)
        infos = [srv.poll(i) for i in ids]
        st = srv.stats()
    assert all(x["done"] and x["status"] == 0 for x in infos)
    assert [x["answer"] for x in infos] == alone
    assert st["completed"] == len(reqs) and st["launches"] >= 1
    assert any(g.n <= 128 for g, *_ in reqs) and any(g.n > 128 for g, *_ in reqs)
    if bit_rows:  # two size classes: n <= 128 on bit-row workers, the rest on CSR walks
        assert st["classes"] == 2 and st["small_max_n"] == 128 and 0 < st["small_workers"] < st["workers"]
    else:         # the default: every request on CSR walkers
        assert st["classes"] == 1 and st["small_max_n"] == 0 and st["small_workers"] == 0


def test_size_class_split_and_small_server(vc):
    # num_workers sets the CSR-walk class's size and the bit-row class gets the slots left; a
    # server for graphs of at most 128 vertices with bit rows is one bit-row class; a split that
    # leaves the bit-row class nothing is an error.
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    reqs = [r for r in mixed_requests(40, 125000) if r[0].n <= 120]
    with vc.Server(max_n=1000, config=vc.make_config(bit_rows=1, num_workers=sms)) as srv:
        st = srv.stats()
        assert st["classes"] == 2 and st["workers"] - st["small_workers"] == sms
    with vc.Server(max_n=120, config=vc.make_config(bit_rows=1)) as srv:
        ids = [srv.submit(g.offsets, g.neighbors, kind, k) for g, kind, k, _ in reqs]
        srv.drain(timeout_ms=120000)
        infos = [srv.poll(i) for i in ids]
        st = srv.stats()
    assert [x["answer"] for x in infos] == [r[3] for r in reqs]
    assert st["classes"] == 1 and st["small_max_n"] == 120 and st["small_workers"] == st["workers"]
    with pytest.raises(vc.VCError):
        vc.Server(max_n=1000, config=vc.make_config(bit_rows=1, num_workers=64 * sms))


def test_trickled_requests_join_a_running_launch(vc):
    reqs = mixed_requests(40, 130000)
    with vc.Server(max_n=1000) as srv:
        ids = []
        for g, kind, k, _ in reqs:
            ids.append(srv.submit(g.offsets, g.neighbors, kind, k))
            time.sleep(0.0005)
        srv.drain(timeout_ms=120000)
        infos = [srv.poll(i) for i in ids]
    assert [x["answer"] for x in infos] == [r[3] for r in reqs]
    assert all(x["submit_ns"] <= x["admit_ns"] <= x["done_ns"] for x in infos)


def test_small_budget_queues_instead_of_failing(vc):
    # A 1 MiB budget leaves a 256 KiB graph arena (about 85 of these graphs): most requests wait
    # in the host queue, and the arena is used up and restarted at least once.
    graphs = [G.gnp(90, 0.07, 140000 + i) for i in range(150)]
    want = [oracle.mvc(g)[0] for g in graphs]
    with vc.Server(max_n=120, budget_bytes=1 << 20) as srv:
        ids = [srv.submit(g.offsets, g.neighbors, 0) for g in graphs]
        srv.drain(timeout_ms=120000)
        got = [srv.poll(i) for i in ids]
        st = srv.stats()
    assert [x["answer"] for x in got] == want
    assert all(x["status"] == 0 for x in got)
    assert st["epochs"] >= 1


def test_rejects_bad_requests(vc):
    with vc.Server(max_n=50) as srv:
        big = G.gnp(60, 0.1, 1)
        with pytest.raises(vc.VCError):
            srv.submit(big.offsets, big.neighbors, 0)
        g = G.cycle(6)
        bad = g.neighbors.copy()
        bad[0] = 4
        with pytest.raises(vc.VCError):
            srv.submit(g.offsets, bad, 0)
        off = g.offsets.copy()
        off[5] = off[6] + 8                 # a later vertex's range runs past the neighbour list
        with pytest.raises(vc.VCError):
            srv.submit(off, g.neighbors, 0)
        rid = srv.submit(g.offsets, g.neighbors, 1, -1)   # k < 0 is answered at once
        assert srv.poll(rid)["done"] == 1 and srv.poll(rid)["answer"] == 0
        rid = srv.submit(g.offsets, g.neighbors, 0)
        srv.drain(timeout_ms=60000)
        assert srv.poll(rid)["answer"] == 3


def test_degenerate_requests(vc):
    # Empty and edgeless graphs, k >= n, k just below and at the minimum, and an empty graph given
    # with null arrays through the C ABI: answers as the definitions give them (MVC(K5) = 4,
    # MVC(P2) = 1, an edgeless graph needs no vertex).
    import ctypes
    empty = G.csr_from_edges(0, [], [])
    edgeless = G.csr_from_edges(6, [], [])
    k5, p2 = G.complete(5), G.path(2)
    cases = [(empty, 0, 0, 0), (empty, 1, 0, 1), (edgeless, 0, 0, 0), (edgeless, 1, 0, 1),
             (k5, 1, 10, 1), (k5, 1, 3, 0), (k5, 0, 0, 4), (p2, 1, 0, 0), (p2, 1, 1, 1)]
    with vc.Server(max_n=50) as srv:
        ids = [srv.submit(g.offsets, g.neighbors, kind, k) for g, kind, k, _ in cases]
        raw = vc.Graph(0, None, None, 0)
        rid = ctypes.c_uint64(0)
        assert srv._lib.vc_server_submit(srv._h, ctypes.byref(raw), 0, 0, ctypes.byref(rid)) == 0
        srv.drain(timeout_ms=60000)
        infos = [srv.poll(i) for i in ids] + [srv.poll(rid.value)]
    assert all(x["done"] and x["status"] == 0 for x in infos)
    assert [x["answer"] for x in infos] == [c[3] for c in cases] + [0]


def test_released_requests_leave_no_records(vc):
    # A long-running server keeps a record per request until the caller releases it: polling with
    # release keeps the held records bounded, and a released id is unknown afterwards.
    reqs = mixed_requests(40, 150000)
    with vc.Server(max_n=1000) as srv:
        held = []
        for rnd in range(5):
            ids = [srv.submit(g.offsets, g.neighbors, kind, k) for g, kind, k, _ in reqs]
            srv.drain(timeout_ms=120000)
            for rid, (_, _, _, want) in zip(ids, reqs):
                info = srv.poll(rid, release=True)
                assert info["done"] == 1 and info["status"] == 0 and info["answer"] == want
            held.append(srv.stats()["records"])
        assert held == [0] * 5
        with pytest.raises(vc.VCError) as e:
            srv.poll(ids[0])
        assert e.value.code == vc.VC_EINVAL
        with pytest.raises(vc.VCError):
            srv.release(ids[0])
        rid = srv.submit(reqs[0][0].offsets, reqs[0][0].neighbors, reqs[0][1], reqs[0][2])
        srv.drain(timeout_ms=120000)
        assert srv.stats()["records"] == 1
        srv.release(rid)
        assert srv.stats()["records"] == 0
