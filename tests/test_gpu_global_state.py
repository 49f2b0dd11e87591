"""GPU parity of the global-memory kernel version (Sec. IV-E): each worker's current node (degree
array, marks, dirty bits, removal list) lives in a private global-memory region instead of shared
memory.  The answers must match the oracle exactly, as for the shared-memory version, and graphs
too large for a shared-memory node must switch to it by themselves.
"""
import numpy as np
import pytest

import oracle
from paper_2204_10402_gb300 import graphs as G
from tests import pins
from tests.test_gpu_parity import check_cover, load_batch_golden, small_graphs

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


def random_state(g, seed, frac=0.15):
    """A seeded intermediate state: a random subset put into S, degrees and m counted plainly."""
    removed = G.uniform01(seed, g.n) < frac
    deg = g.degrees().astype(np.int64)
    src, dst = g.edges()
    m = 0
    for a, b in zip(src.tolist(), dst.tolist()):
        if removed[a] or removed[b]:
            if not removed[a]:
                deg[a] -= 1
            if not removed[b]:
                deg[b] -= 1
        else:
            m += 1
    deg[removed] = -1
    return deg, int(removed.sum()), m


@pytest.mark.parametrize("width,wt", [(16, 32), (32, 128), (16, 512)])
def test_global_reduce_node_random_states(vc, width, wt):
    for i, g in enumerate(small_graphs(24, 21000, 10, 150)):
        deg, S, m = random_state(g, 31000 + i)
        for problem, bound in ((oracle.MVC, S + 6 + i % 9), (oracle.PVC, S + 4 + i % 7)):
            for rules in (1, 2, 4, 7):
                want = oracle.reduce_node(g, deg, S, m, problem, bound, rules)
                got = vc.reduce_node(g.offsets, g.neighbors, deg, S, m, problem, bound, rules,
                                     config=vc.make_config(width=width, worker_threads=wt, node_in_global=1))
                assert got[0].tolist() == want[0].tolist(), (i, problem, rules)
                assert got[1:] == want[1:], (i, problem, rules, got[1:], want[1:])


@pytest.mark.parametrize("width,wt", [(16, 32), (32, 64), (16, 256)])
def test_global_mvc_matches_oracle(vc, width, wt):
    cfg = vc.make_config(width=width, worker_threads=wt, node_in_global=1)
    for g in small_graphs(20, 52000, 4, 90):
        want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors, config=cfg)
        assert a.value == want, (g.n, g.m)
        assert a.stats["node_in_global"] == 1
        check_cover(g, a.cover, want)


def test_global_pvc_around_minimum(vc):
    cfg = vc.make_config(node_in_global=1, worker_threads=64)
    for g in small_graphs(16, 61000, 6, 60):
        best, _, _ = oracle.mvc(g)
        for k in (best - 1, best, best + 1):
            a = vc.pvc(g.offsets, g.neighbors, k, config=cfg)
            assert bool(a.value) == (k >= best), (g.n, g.m, k, best)
            if a.value:
                assert a.cover_size <= k
                check_cover(g, a.cover, a.cover_size)


@pytest.mark.parametrize("cfg", [
    dict(donate_threshold=-1.0),                    # all-local-stack path
    dict(worklist_capacity=1, donate_threshold=1.0),
    dict(num_workers=3, worklist_capacity=2),
])
def test_global_worklist_stress(vc, cfg):
    c = vc.make_config(node_in_global=1, worker_threads=128, **cfg)
    for g in small_graphs(8, 81000, 40, 100):
        want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors, config=c)
        assert a.value == want
        check_cover(g, a.cover, want)


def test_global_batch_matches_stored_answers(vc):
    b = G.batch_gnp(512)
    want = load_batch_golden()
    sizes, covers, st = vc.mvc_batch(b.vtx, b.edge, b.offsets, b.neighbors,
                                     config=vc.make_config(node_in_global=1, worker_threads=64))
    assert st["node_in_global"] == 1
    for i, g in enumerate(b.graphs):
        assert sizes[i] == want[i][2], i
        check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want[i][2])


def test_global_and_shared_agree_on_chung_lu(vc):
    g = G.chung_lu(2000, 6.0, 0)
    best, _, _ = oracle.mvc(g)
    for placement in (-1, 1):
        a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(node_in_global=placement))
        assert a.value == best
        assert a.stats["node_in_global"] == (placement == 1)
        check_cover(g, a.cover, best)


def large_union(tree_n=33000, seed=5):
    """A random tree (solved by the rules; textbook answer) next to a small G(n,p) component that
    needs branching (oracle answer); the cover of a disjoint union adds up."""
    parent = G.random_tree_parents(tree_n, seed)
    tree = G.random_tree(tree_n, seed)
    hard = G.gnp(40, 0.15, seed)
    want = pins.tree_mvc(parent) + oracle.mvc(hard)[0]
    return G.disjoint_union(hard, tree), want


def test_large_graph_switches_to_global_memory(vc):
    # n > 32768 needs 32-bit entries, and a 32-bit node of that size does not fit in shared memory.
    g, want = large_union()
    assert g.n > 32768
    a = vc.mvc(g.offsets, g.neighbors)
    assert a.value == want
    assert a.stats["node_in_global"] == 1 and a.stats["width"] == 32
    check_cover(g, a.cover, want)
    for k, yes in ((want, 1), (want - 1, 0)):
        p = vc.pvc(g.offsets, g.neighbors, k)
        assert p.value == yes
        if yes:
            check_cover(g, p.cover, p.cover_size)
    with pytest.raises(vc.VCError):
        vc.mvc(g.offsets, g.neighbors, config=vc.make_config(node_in_global=-1))
