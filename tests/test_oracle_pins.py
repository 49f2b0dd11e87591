"""Pins for the CPU oracle: every check compares it with something other than itself.

- closed forms: path floor(n/2), cycle ceil(n/2), K_n n-1, K_{a,b} min(a,b), star 1, Petersen 6
- brute-force subset enumeration on random G(n, p), n <= 16
- König's theorem on random bipartite graphs (maximum matching, scipy)
- maximum clique of the complement graph (networkx) on denser graphs
- disjoint-union additivity
- PVC: no at MVC-1, yes at MVC and MVC+1 (Sec. II-A definition of PVC)
- greedy >= MVC >= any maximal matching; every returned cover verifies edge by edge
- hand-derived reduction-rule cases in tests/golden/rules.txt (Sec. II-B, IV-D)
"""
import numpy as np
import pytest

import oracle
from paper_2204_10402_gb300 import graphs as G
from tests import pins

NAMED = [
    *[(f"path{n}", lambda n=n: G.path(n), n // 2) for n in range(1, 13)],
    *[(f"cycle{n}", lambda n=n: G.cycle(n), (n + 1) // 2) for n in range(3, 13)],
    *[(f"K{n}", lambda n=n: G.complete(n), max(n - 1, 0)) for n in range(1, 11)],
    *[(f"K{a},{b}", lambda a=a, b=b: G.complete_bipartite(a, b), min(a, b))
      for a, b in [(1, 1), (2, 3), (3, 3), (3, 7), (5, 4), (6, 6)]],
    *[(f"star{r}", lambda r=r: G.star(r), 1) for r in (1, 2, 5, 12)],
    ("petersen", G.petersen, 6),
]


def random_small_graphs(count=60, seed0=1000):
    out = []
    for i in range(count):
        u = G.uniform01(seed0 + i, 2, 0)
        n = 4 + int(u[0] * 13)  # 4..16
        p = [0.1, 0.2, 0.3, 0.5, 0.7][i % 5]
        out.append(G.gnp(n, p, seed0 + i, draw_offset=2))
    return out


def run_pins(orc, quick=False):
    """Runs the pin battery against one oracle build; returns a list of failure descriptions."""
    fails = []
    for name, make, want in NAMED:
        g = make()
        got, cover, _ = orc.mvc(g)
        if got != want:
            fails.append(f"{name}: mvc {got} != closed form {want}")
        elif cover.sum() != want or not oracle.verify_cover(g, cover):
            fails.append(f"{name}: cover invalid")
    for g in random_small_graphs(24 if quick else 60):
        want = pins.brute_force_mvc(g)
        got, cover, _ = orc.mvc(g)
        if got != want:
            fails.append(f"G({g.n}) m={g.m}: mvc {got} != brute force {want}")
            continue
        if cover.sum() != want or not oracle.verify_cover(g, cover):
            fails.append(f"G({g.n}) m={g.m}: cover invalid")
        for k, yes in ((want - 1, False), (want, True), (want + 1, True)):
            found, c, _ = orc.pvc(g, k)
            if found != yes:
                fails.append(f"G({g.n}) m={g.m}: pvc(k={k}) {found}, MVC {want}")
            elif found and (c.sum() > k or not oracle.verify_cover(g, c)):
                fails.append(f"G({g.n}) m={g.m}: pvc(k={k}) cover invalid")
    for case in pins.load_rule_cases():
        g = G.csr_from_edges(case["n"], [e[0] for e in case["edges"]], [e[1] for e in case["edges"]])
        deg = case.get("start_deg", g.degrees().tolist())
        d, S, m, pruned = orc.reduce_node(g, deg, case.get("start_S", 0), case.get("start_m", g.m),
                                          case["mode"], case["bound"], case["rules"])
        got = (d.tolist(), S, m, int(pruned))
        want = (case["expect_deg"], case["expect_S"], case["expect_m"], case["expect_pruned"])
        if got != want:
            fails.append(f"rule case {case['name']}: {got} != {want}")
    for case in pins.load_greedy_cases():
        g = G.csr_from_edges(case["n"], [e[0] for e in case["edges"]], [e[1] for e in case["edges"]])
        size, cover = orc.greedy(g)
        got = (size, sorted(int(v) for v in np.flatnonzero(cover)))
        want = (case["expect_greedy"], case["expect_cover"])
        if got != want:
            fails.append(f"greedy case {case['name']}: {got} != {want}")
    return fails


def test_pin_battery():
    fails = run_pins(oracle._default())
    assert not fails, "\n".join(fails)


@pytest.mark.parametrize("seed", range(12))
def test_konig_bipartite(seed):
    u = G.uniform01(5000 + seed, 3)
    a, b = 5 + int(u[0] * 30), 5 + int(u[1] * 30)
    p = 0.04 + 0.2 * u[2]
    g = G.random_bipartite(a, b, p, 5000 + seed)
    want = pins.konig_mvc(g, a)
    got, cover, _ = oracle.mvc(g)
    assert got == want
    assert cover.sum() == got and oracle.verify_cover(g, cover)


@pytest.mark.parametrize("seed", range(8))
def test_complement_clique(seed):
    n = 22 + 2 * seed
    g = G.gnp(n, 0.35 + 0.05 * (seed % 4), 7000 + seed)
    want = pins.complement_clique_mvc(g)
    got, cover, _ = oracle.mvc(g)
    assert got == want
    assert oracle.verify_cover(g, cover)


def test_disjoint_union_additivity():
    parts = [G.gnp(14, 0.3, 11), G.petersen(), G.cycle(9), G.gnp(18, 0.2, 12)]
    total = parts[0]
    want = oracle.mvc(parts[0])[0]
    for p in parts[1:]:
        total = G.disjoint_union(total, p)
        want += oracle.mvc(p)[0]
    assert oracle.mvc(total)[0] == want


@pytest.mark.parametrize("seed", range(6))
def test_tree_dynamic_programme(seed):
    # Trees: the rules alone solve them, and the answer has a textbook dynamic programme.
    for n in (1, 2, 9, 40, 300):
        parent = G.random_tree_parents(n, seed * 1000 + n)
        g = G.random_tree(n, seed * 1000 + n)
        want = pins.tree_mvc(parent)
        if n <= 20:
            assert pins.brute_force_mvc(g) == want
        assert oracle.mvc(g)[0] == want
        assert oracle.greedy(g)[0] == want


def test_greedy_bounds_and_covers():
    for g in random_small_graphs(40, seed0=3000) + [G.gnp(60, 0.1, 0), G.gnp(120, 0.05, 4)]:
        gs, gc = oracle.greedy(g)
        assert oracle.verify_cover(g, gc) and gc.sum() == gs
        best, cover, stats = oracle.mvc(g)
        assert gs >= best >= pins.maximal_matching_size(g)
        assert stats["greedy"] == gs
        assert oracle.verify_cover(g, cover) and cover.sum() == best


def test_edge_cases():
    empty = G.csr_from_edges(0, [], [])
    assert oracle.mvc(empty)[0] == 0
    isolated = G.csr_from_edges(7, [], [])
    assert oracle.mvc(isolated)[0] == 0
    assert oracle.pvc(isolated, 0)[0] is True
    g = G.petersen()
    assert oracle.pvc(g, -1)[0] is False
    assert oracle.pvc(g, g.n)[0] is True
    assert oracle.pvc(G.csr_from_edges(3, [], []), -1)[0] is False


def test_pvc_matches_mvc_on_medium_graphs():
    # PVC(k) is yes iff k >= MVC (Sec. II-A); checked across the threshold on searched graphs.
    for seed in range(6):
        g = G.gnp(45, 0.12, 9000 + seed)
        best = oracle.mvc(g)[0]
        assert oracle.pvc(g, best - 1)[0] is False
        found, c, _ = oracle.pvc(g, best)
        assert found and c.sum() <= best and oracle.verify_cover(g, c)


def test_config1_answer():
    # G(60, 0.10), seed 0: the first workload of the benchmark family; answer pinned by the
    # complement-clique solver (an independent exact method).
    g = G.gnp(60, 0.10, 0)
    got, cover, _ = oracle.mvc(g)
    assert got == pins.complement_clique_mvc(g)
    assert oracle.verify_cover(g, cover)
