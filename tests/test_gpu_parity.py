"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

All answers are integers and must match exactly: MVC size, PVC yes/no, the greedy bound, and the
reduced degree array of a single node (the rule passes are deterministic rounds, Sec. IV-D
tie-breaks).  Every cover the GPU returns must verify edge by edge and have the reported size.
Node counts are not compared (the parallel search order differs from the oracle's).
"""
import numpy as np
import pytest

import oracle
from paper_2204_10402_gb300 import graphs as G
from tests import pins

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


def small_graphs(count, seed0, n_lo=4, n_hi=40):
    out = []
    for i in range(count):
        u = G.uniform01(seed0 + i, 2)
        n = n_lo + int(u[0] * (n_hi - n_lo + 1))
        p = [0.05, 0.1, 0.2, 0.3, 0.5, 0.8][i % 6]
        out.append(G.gnp(n, p, seed0 + i, draw_offset=2))
    return out


def check_cover(g, cover, size):
    c = np.asarray(cover).astype(bool)[: g.n]
    assert c.sum() == size
    assert oracle.verify_cover(g, c)


# ------------------------------------------------------------------------------------------------
# single-node reduction: bit-exact degree arrays
# ------------------------------------------------------------------------------------------------

def test_rule_golden_cases(vc):
    for case in pins.load_rule_cases():
        g = G.csr_from_edges(case["n"], [e[0] for e in case["edges"]], [e[1] for e in case["edges"]])
        deg = case.get("start_deg", g.degrees().tolist())
        for width in (16, 32):
            cfg = vc.make_config(width=width)
            d, S, m, pruned = vc.reduce_node(g.offsets, g.neighbors, deg, case.get("start_S", 0),
                                             case.get("start_m", g.m), case["mode"], case["bound"],
                                             case["rules"], config=cfg)
            got = (d.tolist(), S, m, int(pruned))
            want = (case["expect_deg"], case["expect_S"], case["expect_m"], case["expect_pruned"])
            assert got == want, (case["name"], width, got, want)


@pytest.mark.parametrize("wt,bit_rows", [(32, 1), (32, -1), (64, 0), (256, 0)])
def test_reduce_node_random_states(vc, wt, bit_rows):
    # bit_rows = 1: adjacency bit rows (graphs up to 256 vertices; larger ones use CSR walks)
    rng_graphs = small_graphs(40, 20000, 10, 250)
    for i, g in enumerate(rng_graphs):
        rows = bit_rows if (bit_rows <= 0 or g.n <= 256) else 0
        # a random intermediate state: remove a seeded subset, then reduce from there
        u = G.uniform01(30000 + i, g.n)
        removed = u < 0.15
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
        S = int(removed.sum())
        for problem, bound in ((oracle.MVC, S + 6 + i % 9), (oracle.PVC, S + 4 + i % 7)):
            for rules in (1, 2, 4, 7):
                want = oracle.reduce_node(g, deg, S, m, problem, bound, rules)
                got = vc.reduce_node(g.offsets, g.neighbors, deg, S, m, problem, bound, rules,
                                     config=vc.make_config(worker_threads=wt, bit_rows=rows))
                assert got[0].tolist() == want[0].tolist(), (i, problem, rules)
                assert got[1:] == want[1:], (i, problem, rules, got[1:], want[1:])


# ------------------------------------------------------------------------------------------------
# greedy bound: same deterministic rounds and tie-breaks, so identical values
# ------------------------------------------------------------------------------------------------

def test_greedy_matches_oracle(vc):
    for g in small_graphs(30, 40000, 5, 200) + [G.gnp(60, 0.1, 0), G.chung_lu(2000, 6.0, 0)]:
        want, _ = oracle.greedy(g)
        got, cover = vc.greedy(g.offsets, g.neighbors)
        assert got == want
        check_cover(g, cover, got)


# ------------------------------------------------------------------------------------------------
# MVC / PVC answers
# ------------------------------------------------------------------------------------------------

def test_mvc_closed_forms(vc):
    cases = [(G.path(n), n // 2) for n in (2, 3, 7, 20)] + [(G.cycle(n), (n + 1) // 2) for n in (3, 4, 9, 31)]
    cases += [(G.complete(n), n - 1) for n in (2, 5, 12)] + [(G.complete_bipartite(4, 9), 4), (G.star(7), 1),
                                                          (G.petersen(), 6)]
    for g, want in cases:
        a = vc.mvc(g.offsets, g.neighbors)
        assert a.value == want
        check_cover(g, a.cover, want)


def test_mvc_random_small(vc):
    for g in small_graphs(60, 50000, 4, 60):
        want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors)
        assert a.value == want, (g.n, g.m)
        check_cover(g, a.cover, want)


def test_pvc_around_minimum(vc):
    for g in small_graphs(30, 60000, 6, 60):
        best, _, _ = oracle.mvc(g)
        for k in (best - 1, best, best + 1):
            a = vc.pvc(g.offsets, g.neighbors, k)
            assert bool(a.value) == (k >= best), (g.n, g.m, k, best)
            if a.value:
                assert a.cover_size <= k
                check_cover(g, a.cover, a.cover_size)


@pytest.mark.parametrize("width,wt,bit_rows", [(16, 32, 0), (32, 32, 0), (16, 32, -1), (32, 32, -1),
                                               (16, 128, 0), (32, 64, 0), (16, 512, 0)])
def test_variants_agree(vc, width, wt, bit_rows):
    for g in small_graphs(12, 70000, 30, 90):
        want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(width=width, worker_threads=wt, bit_rows=bit_rows))
        assert a.value == want
        assert a.stats["bit_rows"] == (0 if bit_rows < 0 or wt > 32 else (2 if g.n <= 64 else 4) if g.n > 32 else 1)
        check_cover(g, a.cover, want)


@pytest.mark.parametrize("cfg", [
    dict(donate_threshold=-1.0),                    # never donate: all-local-stack path
    dict(worklist_capacity=1, donate_threshold=1.0),
    dict(donate_threshold=1.0),                     # donate whenever the ring has room
    dict(num_workers=1),                            # one worker
    dict(num_workers=3, worklist_capacity=2),
])
def test_worklist_stress(vc, cfg):
    for g in small_graphs(10, 80000, 40, 100):
        want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(**cfg))
        assert a.value == want
        check_cover(g, a.cover, want)


def test_device_tensor_inputs(vc):
    import torch
    for g in small_graphs(8, 90000, 20, 80):
        want, _, _ = oracle.mvc(g)
        off = torch.from_numpy(g.offsets).cuda()
        nbr = torch.from_numpy(g.neighbors).cuda()
        a = vc.mvc(off, nbr)
        assert a.value == want
        assert a.cover.is_cuda
        check_cover(g, a.cover.cpu().numpy(), want)
        p = vc.pvc(off, nbr, want - 1)
        assert p.value == 0


def test_edge_cases(vc):
    empty = G.csr_from_edges(0, [], [])
    assert vc.mvc(empty.offsets, empty.neighbors).value == 0
    iso = G.csr_from_edges(9, [], [])
    a = vc.mvc(iso.offsets, iso.neighbors)
    assert a.value == 0 and a.cover.sum() == 0
    assert vc.pvc(iso.offsets, iso.neighbors, 0).value == 1
    g = G.petersen()
    assert vc.pvc(g.offsets, g.neighbors, -1).value == 0
    assert vc.pvc(g.offsets, g.neighbors, g.n + 5).value == 1
    one = G.path(2)
    assert vc.mvc(one.offsets, one.neighbors).value == 1


def test_invalid_csr_rejected(vc):
    g = G.cycle(6)
    bad = g.neighbors.copy()
    bad[0] = 5 if bad[0] != 5 else 4    # breaks symmetry / order
    with pytest.raises(vc.VCError) as e:
        vc.mvc(g.offsets, bad)
    assert e.value.code == vc.VC_EINVAL
    loop = G.csr_from_edges(3, [0, 1], [1, 2])
    nb = loop.neighbors.copy()
    nb[0] = 0                            # self-loop
    with pytest.raises(vc.VCError):
        vc.mvc(loop.offsets, nb)
    off = g.offsets.copy()
    off[2] = off[3] + 1                  # offsets not monotone
    with pytest.raises(vc.VCError):
        vc.mvc(off, g.neighbors)
    # the library stays usable after a rejected call
    assert vc.mvc(g.offsets, g.neighbors).value == 3


def test_idle_timeout_reports_status(vc):
    # A tiny idle limit makes idle workers give up while one worker still searches: the call must
    # return VC_ETIMEOUT (not hang, not fault) and the next call must work normally.
    g = G.gnp(110, 0.12, 123)
    with pytest.raises(vc.VCError) as e:
        vc.mvc(g.offsets, g.neighbors, config=vc.make_config(idle_timeout_ns=1, donate_threshold=-1.0))
    assert e.value.code == vc.VC_ETIMEOUT
    want, _, _ = oracle.mvc(g)
    assert vc.mvc(g.offsets, g.neighbors).value == want


# ------------------------------------------------------------------------------------------------
# the benchmark workloads
# ------------------------------------------------------------------------------------------------

def test_config_gnp60(vc):
    g = G.gnp(60, 0.10, 0)
    want, _, _ = oracle.mvc(g)
    a = vc.mvc(g.offsets, g.neighbors)
    assert a.value == want
    check_cover(g, a.cover, want)


def test_config_chung_lu_2000_pvc(vc):
    # Table I's PVC columns: k = min (yes), k = min - 1 (no: the whole tree), k = min + 1 (yes).
    g = G.chung_lu(2000, 6.0, 0)
    best, _, _ = oracle.mvc(g)
    yes = vc.pvc(g.offsets, g.neighbors, best)
    no = vc.pvc(g.offsets, g.neighbors, best - 1)
    assert yes.value == 1 and no.value == 0
    check_cover(g, yes.cover, yes.cover_size)
    assert yes.cover_size <= best
    above = vc.pvc(g.offsets, g.neighbors, best + 1)
    assert above.value == 1 and above.cover_size <= best + 1
    check_cover(g, above.cover, above.cover_size)
    m = vc.mvc(g.offsets, g.neighbors)
    assert m.value == best


@pytest.mark.parametrize("n", [120, 160])
@pytest.mark.parametrize("width", [16, 32])
def test_config_planted_clique_family(vc, n, width):
    g, _ = G.gnp_with_planted_clique(n, 0.05, round(25 * n / 400), 0)
    want, _, _ = oracle.mvc(g)
    a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(width=width))
    assert a.value == want
    check_cover(g, a.cover, want)


def test_batch_matches_oracle(vc):
    b = G.batch_gnp(256)
    sizes, covers, st = vc.mvc_batch(b.vtx, b.edge, b.offsets, b.neighbors)
    for i, g in enumerate(b.graphs):
        want, _, _ = oracle.mvc(g)
        assert sizes[i] == want, i
        check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want)
    assert st["nodes_visited"] > 0


@pytest.mark.parametrize("bit_rows", [1, -1])
def test_batch_adjacency_modes_match_stored_answers(vc, bit_rows):
    # The bench batch's first 512 graphs with bit rows forced on and off.
    b = G.batch_gnp(512)
    want = load_batch_golden()
    sizes, covers, st = vc.mvc_batch(b.vtx, b.edge, b.offsets, b.neighbors, config=vc.make_config(bit_rows=bit_rows))
    assert st["bit_rows"] == (4 if bit_rows > 0 else 0)
    for i, g in enumerate(b.graphs):
        assert sizes[i] == want[i][2], i
        check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want[i][2])


def mid_size_graphs():
    # 129-256 vertices (eight-word bit rows by default), trees the oracle finishes in under a second
    out = [G.gnp(n, p, s) for n, p, s in [(140, 0.04, 11), (180, 0.025, 12), (230, 0.018, 13), (256, 0.015, 14),
                                          (129, 0.05, 15)]]
    out += [G.chung_lu(200, 6.0, 21), G.chung_lu(256, 9.0, 22)]
    out.append(G.gnp_with_planted_clique(140, 0.05, 9, 0)[0])
    return out


@pytest.mark.parametrize("width", [32, 16])
def test_mid_size_graphs_default_bit_rows(vc, width):
    # The default workers for 129-256 vertices (eight-word rows) against the oracle, MVC and PVC at
    # k = MVC - 1 / MVC, and against CSR walks (bit_rows = -1) on the same graphs.
    for g in mid_size_graphs():
        want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(width=width))
        assert a.stats["bit_rows"] == 8, g.n
        assert a.value == want, (g.n, g.m)
        check_cover(g, a.cover, want)
        csr = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(width=width, bit_rows=-1))
        assert csr.stats["bit_rows"] == 0 and csr.value == want
        for k in (want - 1, want):
            p = vc.pvc(g.offsets, g.neighbors, k, config=vc.make_config(width=width))
            assert p.value == (1 if k >= want else 0), (g.n, k)
            if p.value:
                check_cover(g, p.cover, p.cover_size)
                assert p.cover_size <= k


def test_mid_size_batch_default_bit_rows(vc):
    # A batch whose largest graph has 129-256 vertices runs on eight-word rows.
    b = G.batch_gnp(64, first_seed=60000, n_lo=129, n_hi=256, p_lo=0.014, p_hi=0.02)
    sizes, covers, st = vc.mvc_batch(b.vtx, b.edge, b.offsets, b.neighbors)
    assert st["bit_rows"] == 8
    for i, g in enumerate(b.graphs):
        want, _, _ = oracle.mvc(g)
        assert sizes[i] == want, i
        check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want)


def load_batch_golden():
    import os
    rows = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096_mvc.txt")
    for line in open(path):
        if line.startswith("#"):
            continue
        g, n, m, size, nodes = (int(x) for x in line.split())
        rows[g] = (n, m, size)
    return rows


def test_full_batch_matches_stored_oracle_answers(vc):
    # The benchmark's launch configuration (defaults, 4096 graphs, device-resident CSR) against the
    # oracle's answers written by tests/golden/make_batch_golden.py; every cover verifies.
    import torch
    b = G.batch_gnp(4096)
    want = load_batch_golden()
    off = torch.from_numpy(b.offsets).cuda()
    nbr = torch.from_numpy(b.neighbors).cuda()
    sizes, covers, st = vc.mvc_batch(b.vtx, b.edge, off, nbr)
    covers = covers.cpu().numpy()
    for i, g in enumerate(b.graphs):
        assert (g.n, g.m) == want[i][:2]
        assert sizes[i] == want[i][2], i
        check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want[i][2])


def _remove(g, deg, S, m, vertices):
    """Puts a set of live vertices into S (Sec. IV-B removal), written out plainly for the test."""
    deg = np.array(deg, dtype=np.int64)
    chosen = set(int(v) for v in vertices)
    for v in chosen:
        for x in g.neighbors[g.offsets[v]:g.offsets[v + 1]].tolist():
            if deg[x] == -1:
                continue
            if x in chosen:
                if x > v:
                    m -= 1
            else:
                deg[x] -= 1
                m -= 1
    for v in chosen:
        deg[v] = -1
    return deg, S + len(chosen), m


@pytest.mark.parametrize("wt,bit_rows", [(32, 0), (32, -1), (128, 0)])
def test_reduce_after_branch_matches_full_reduction(vc, wt, bit_rows):
    # The traversal re-examines only vertices whose degree changed after a branch.  From a fixpoint
    # state, put v (or N(v)) into S and reduce: the result must equal the oracle's full reduction
    # of the same child state.
    cfg = vc.make_config(worker_threads=wt, bit_rows=bit_rows)
    for i, g in enumerate(small_graphs(30, 110000, 20, 150)):
        for problem, slack in ((oracle.MVC, 40), (oracle.PVC, 30)):
            bound = min(g.n, int(0.6 * g.n) + slack % 7)
            P, S, m, pruned = oracle.reduce_node(g, g.degrees(), 0, g.m, problem, bound, 7)
            if pruned or m == 0:
                continue
            live = [v for v in range(g.n) if P[v] > 0]
            for v in live[:: max(1, len(live) // 4)]:
                nb = [x for x in g.neighbors[g.offsets[v]:g.offsets[v + 1]].tolist() if P[x] != -1]
                for branch, chosen in ((v, [v]), (-2 - v, nb)):
                    child, S1, m1 = _remove(g, P, S, m, chosen)
                    want = oracle.reduce_node(g, child, S1, m1, problem, bound, 7)
                    got = vc.reduce_node(g.offsets, g.neighbors, P, S, m, problem, bound, 7, config=cfg,
                                         branch=branch)
                    assert got[0].tolist() == want[0].tolist(), (i, v, branch)
                    assert got[1:] == want[1:], (i, v, branch, got[1:], want[1:])


@pytest.mark.parametrize("wt", [64, 128])
def test_batch_multiwarp_workers(vc, wt):
    # Workers of several warps on many graphs: every warp must finish reading a node before any
    # warp loads the next one (a race here desynchronises the block's barriers).
    import torch
    b = G.batch_gnp(1024)
    want = load_batch_golden()
    off = torch.from_numpy(b.offsets).cuda()
    nbr = torch.from_numpy(b.neighbors).cuda()
    for _ in range(2):
        sizes, covers, st = vc.mvc_batch(b.vtx, b.edge, off, nbr, config=vc.make_config(worker_threads=wt))
        assert st["worker_threads"] == wt
        assert [int(x) for x in sizes] == [want[i][2] for i in range(1024)]


def test_batch_with_degenerate_members(vc):
    # A ragged batch: empty and edgeless graphs, a single edge, closed forms and ordinary graphs
    # side by side (through vc_mvc_batch and a batch plan); batches of one graph, of empty graphs
    # only, and of no graph.
    import torch
    empty = G.csr_from_edges(0, [], [])
    members = [empty, G.csr_from_edges(7, [], []), G.path(2), G.petersen(), G.gnp(60, 0.10, 0), empty,
               G.complete(5), G.star(8), G.gnp(120, 0.3, 7, draw_offset=2), G.csr_from_edges(1, [], [])]
    want = [oracle.mvc(g)[0] for g in members]
    assert want[:4] == [0, 0, 1, 6] and want[6:8] == [4, 1]
    b = G.pack(members)
    sizes, covers, _ = vc.mvc_batch(b.vtx, b.edge, b.offsets, b.neighbors)
    assert [int(x) for x in sizes] == want
    for i, g in enumerate(members):
        check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want[i])
    plan = vc.BatchPlan(b.vtx, b.edge, torch.from_numpy(b.offsets).cuda(), torch.from_numpy(b.neighbors).cuda())
    plan.launch()
    psizes, pcovers, _ = plan.results(want_covers=True)
    plan.close()
    assert [int(x) for x in psizes] == want
    for i, g in enumerate(members):
        check_cover(g, pcovers[b.vtx[i]: b.vtx[i + 1]], want[i])
    for group in ([G.petersen()], [empty], [empty, G.csr_from_edges(3, [], []), empty]):
        pb = G.pack(group)
        s2, c2, _ = vc.mvc_batch(pb.vtx, pb.edge, pb.offsets, pb.neighbors)
        assert [int(x) for x in s2] == [oracle.mvc(g)[0] for g in group]
    s0, _, _ = vc.mvc_batch(np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(0, np.int32),
                            np.zeros(0, np.int32))
    assert s0.size == 0


def test_batch_plan_graph_replay(vc):
    # The batch captured as one CUDA graph, replayed three times: identical answers every time,
    # equal to the oracle's, with valid covers.
    import torch
    b = G.batch_gnp(512)
    want = load_batch_golden()
    plan = vc.BatchPlan(b.vtx, b.edge, torch.from_numpy(b.offsets).cuda(), torch.from_numpy(b.neighbors).cuda())
    for _ in range(3):
        plan.launch()
        sizes, covers, st = plan.results(want_covers=True)
        assert [int(x) for x in sizes] == [want[i][2] for i in range(512)]
        for i, g in enumerate(b.graphs[:64]):
            check_cover(g, covers[b.vtx[i]: b.vtx[i + 1]], want[i][2])
        assert st["nodes_visited"] > 0 and st["kernel_ms"] > 0
    plan.close()
    bad = G.cycle(5)
    nb = bad.neighbors.copy()
    nb[0] = 3
    pb = G.pack([bad])
    with pytest.raises(vc.VCError):
        vc.BatchPlan(pb.vtx, pb.edge, pb.offsets, nb)


def test_batch_plan_completion_times(vc):
    # When each graph of a launch was answered: MVC needs a search for every graph with an edge
    # (the greedy bound alone proves no minimum), so each answer comes after the greedy pass began
    # and within the launch; the largest search (oracle nodes) ends no earlier than the median graph.
    import os
    import torch
    b = G.batch_gnp(512)
    plan = vc.BatchPlan(b.vtx, b.edge, torch.from_numpy(b.offsets).cuda(), torch.from_numpy(b.neighbors).cuda())
    plan.launch()
    sizes, _, st = plan.results()
    t = plan.completion_ms()
    plan.close()
    assert t.shape == (512,) and (t >= 0).all()
    has_edges = np.array([g.m > 0 for g in b.graphs])
    assert (t[has_edges] > 0).all()
    assert t.max() <= st["kernel_ms"] + 5.0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096_mvc.txt")
    nodes = np.array([int(l.split()[4]) for l in open(path) if not l.startswith("#")][:512])
    assert t[int(np.argmax(nodes))] >= np.median(t)


def load_clique_golden():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "planted_clique_mvc.txt")
    rows = {}
    for line in open(path):
        if not line.startswith("#"):
            n, c, m, size, nodes, secs = line.split()
            rows[int(n)] = (int(c), int(m), int(size))
    return rows


def test_planted_clique_pvc_three_columns(vc):
    # Table I's three PVC instances (k = min-1, min, min+1) on the planted-clique family.
    g, _ = G.gnp_with_planted_clique(160, 0.05, 10, 0)
    best, _, _ = oracle.mvc(g)
    for k in (best - 1, best, best + 1):
        a = vc.pvc(g.offsets, g.neighbors, k)
        assert bool(a.value) == (k >= best)
        if a.value:
            check_cover(g, a.cover, a.cover_size)
            assert a.cover_size <= k


@pytest.mark.parametrize("n,bit_rows", [(180, 1), (200, 0), (180, -1), (200, -1)])
def test_planted_clique_stored_answers(vc, n, bit_rows):
    # Sizes the oracle needs minutes for (answers stored by tests/golden/make_clique_golden.py);
    # 8-word bit rows by default and on request (bit_rows = 1), CSR walks with bit_rows = -1.
    c, m, want = load_clique_golden()[n]
    g, _ = G.gnp_with_planted_clique(n, 0.05, c, 0)
    assert g.m == m
    a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(bit_rows=bit_rows))
    assert a.value == want
    assert a.stats["bit_rows"] == (0 if bit_rows < 0 else 8)
    check_cover(g, a.cover, want)
    assert vc.pvc(g.offsets, g.neighbors, want - 1, want_cover=False).value == 0


def test_per_sm_load_counts(vc):
    # Sec. V-C load measure: every SM expands tree nodes and the counts add up to the total.
    b = G.batch_gnp(1024)
    sizes, _, st = vc.mvc_batch(b.vtx, b.edge, b.offsets, b.neighbors, want_covers=False)
    per_sm = vc.last_sm_nodes()
    assert per_sm.sum() == st["nodes_visited"]
    assert (per_sm > 0).sum() >= 100


def test_l2_copy_probe(vc):
    # The roofline's L2 probe: after p passes dst holds src with the pass index p-1 folded into
    # the first word of every 16 bytes.
    import torch
    src = torch.arange(1 << 16, dtype=torch.int32, device="cuda")
    dst = torch.zeros_like(src)
    vc.l2_copy_probe(dst, src, 3)
    torch.cuda.synchronize()
    want = src.clone().view(-1, 4)
    want[:, 0] ^= 2
    assert torch.equal(dst.view(-1, 4), want)
    with pytest.raises(vc.VCError):
        vc.l2_copy_probe(dst[1:], src[1:], 1)  # not 16-byte aligned


def boundary_graphs():
    """Graphs at the bit-row word boundaries (32, 64, 128, 256 vertices and one either side), with
    closed-form answers or small enough for the oracle."""
    cases = [(G.complete(n), n - 1) for n in (31, 32, 33)]
    cases += [(G.path(n), n // 2) for n in (63, 64, 65)] + [(G.cycle(n), (n + 1) // 2) for n in (127, 128, 129)]
    cases += [(G.star(n - 1), 1) for n in (255, 256)] + [(G.complete_bipartite(16, 48), 16)]
    for n, p in ((1, 0.5), (2, 1.0), (3, 0.7), (31, 0.2), (33, 0.3), (63, 0.1), (65, 0.12), (127, 0.05),
                 (128, 0.06), (129, 0.04), (200, 0.02), (256, 0.015)):
        g = G.gnp(n, p, 7000 + n)
        cases.append((g, None))
    return cases


@pytest.mark.parametrize("bit_rows", [1, -1])
def test_bit_row_size_boundaries(vc, bit_rows):
    for g, want in boundary_graphs():
        if want is None:
            want, _, _ = oracle.mvc(g)
        a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(bit_rows=bit_rows))
        assert a.value == want, (g.n, g.m)
        words = 0 if bit_rows < 0 else (1 if g.n <= 32 else 2 if g.n <= 64 else 4 if g.n <= 128 else 8)
        assert a.stats["bit_rows"] == words, g.n
        check_cover(g, a.cover, want)
        p = vc.pvc(g.offsets, g.neighbors, want - 1, config=vc.make_config(bit_rows=bit_rows))
        assert p.value == 0  # no cover below the minimum (and k = -1 is always no)


def test_bit_rows_rejected_where_they_cannot_run(vc):
    # Bit rows need one-warp workers with the node in shared memory and n <= 256.
    g = G.gnp(60, 0.1, 0)
    for cfg in (dict(bit_rows=1, worker_threads=64), dict(bit_rows=1, node_in_global=1)):
        with pytest.raises(vc.VCError):
            vc.mvc(g.offsets, g.neighbors, config=vc.make_config(**cfg))
    big = G.gnp(300, 0.02, 1)
    with pytest.raises(vc.VCError):
        vc.mvc(big.offsets, big.neighbors, config=vc.make_config(bit_rows=1, worker_threads=32))
    # auto mode falls back to CSR walks in the same cases
    a = vc.mvc(g.offsets, g.neighbors, config=vc.make_config(worker_threads=64))
    assert a.stats["bit_rows"] == 0 and a.value == oracle.mvc(g)[0]


def test_cancel_flag_stops_a_running_search(vc):
    # The caller's cancel flag (device or host memory) ends even a search whose workers never go
    # idle; the library answers normally afterwards.
    import threading
    import time

    import torch
    c, m, want = load_clique_golden()[200]
    g, _ = G.gnp_with_planted_clique(200, 0.05, c, 0)
    t0 = time.time()
    full = vc.mvc(g.offsets, g.neighbors, want_cover=False)
    full_s = time.time() - t0
    assert full.value == want
    flag = torch.ones(1, dtype=torch.int32, device="cuda")  # raised before the call
    with pytest.raises(vc.VCError) as e:
        vc.mvc(g.offsets, g.neighbors, config=vc.make_config(cancel=flag.data_ptr()))
    assert e.value.code == -6  # VC_ECANCELLED
    host_flag = torch.zeros(1, dtype=torch.int32).pin_memory()  # raised by the host mid-search
    timer = threading.Timer(0.05, lambda: host_flag.fill_(1))
    t0 = time.time()
    timer.start()
    with pytest.raises(vc.VCError) as e:
        vc.mvc(g.offsets, g.neighbors, config=vc.make_config(cancel=host_flag.data_ptr()))
    timer.join()
    assert e.value.code == -6
    assert time.time() - t0 < 0.5 * full_s
    small = G.gnp(60, 0.1, 0)
    assert vc.mvc(small.offsets, small.neighbors).value == oracle.mvc(small)[0]
