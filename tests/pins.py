"""Independent checks that pin the oracle.  Nothing here calls the oracle or the CUDA path.

- brute_force_mvc: exhaustive subset enumeration (the definition of a minimum vertex cover).
- konig_mvc: for bipartite graphs the minimum cover size equals the maximum matching size
  (König's theorem); the matching comes from scipy's Hopcroft-Karp routine.
- complement_clique_mvc: the complement of a minimum cover is a maximum independent set, i.e. a
  maximum clique of the complement graph; the clique comes from networkx.
- maximal_matching_size: any maximal matching is a lower bound on the cover size.
- tree_mvc: the textbook dynamic programme over a rooted tree (each vertex either in the cover,
  or out of it with all its children in).
- load_rule_cases: parses tests/golden/rules.txt.
- load_greedy_cases: parses tests/golden/greedy.txt (hand-derived greedy bounds and covers).
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def brute_force_mvc(g) -> int:
    assert g.n <= 22, "brute force is for tiny graphs"
    u, v = g.edges()
    if u.size == 0:
        return 0
    masks = np.arange(1 << g.n, dtype=np.int64)
    ok = np.ones(masks.size, dtype=bool)
    for a, b in zip(u.tolist(), v.tolist()):
        ok &= (((masks >> a) | (masks >> b)) & 1).astype(bool)
    pop = np.zeros(masks.size, dtype=np.int64)
    for bit in range(g.n):
        pop += (masks >> bit) & 1
    return int(pop[ok].min())


def konig_mvc(g, left: int) -> int:
    import scipy.sparse as sp
    from scipy.sparse.csgraph import maximum_bipartite_matching
    u, v = g.edges()
    right = g.n - left
    if u.size == 0:
        return 0
    biadj = sp.csr_matrix((np.ones(u.size), (u, v - left)), shape=(left, right))
    match = maximum_bipartite_matching(biadj, perm_type="column")
    return int((match >= 0).sum())


def complement_clique_mvc(g) -> int:
    import networkx as nx
    h = nx.complete_graph(g.n)
    u, v = g.edges()
    h.remove_edges_from(zip(u.tolist(), v.tolist()))
    clique, _ = nx.max_weight_clique(h, weight=None)
    return g.n - len(clique)


def tree_mvc(parent: np.ndarray) -> int:
    """Minimum cover of the forest given by parent[] (parent[v] < v, roots have -1)."""
    n = len(parent)
    take = np.ones(n, dtype=np.int64)   # v in the cover: 1 + sum over children of the better choice
    skip = np.zeros(n, dtype=np.int64)  # v not in the cover: every child is in it
    for v in range(n - 1, -1, -1):
        p = int(parent[v])
        if p >= 0:
            take[p] += min(take[v], skip[v])
            skip[p] += take[v]
    roots = np.nonzero(parent < 0)[0]
    return int(sum(min(take[r], skip[r]) for r in roots))


def maximal_matching_size(g) -> int:
    used = np.zeros(g.n, dtype=bool)
    size = 0
    u, v = g.edges()
    for a, b in zip(u.tolist(), v.tolist()):
        if not used[a] and not used[b]:
            used[a] = used[b] = True
            size += 1
    return size


def load_rule_cases(path: str | None = None) -> list:
    path = path or os.path.join(GOLDEN, "rules.txt")
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "case":
                cur = {"name": rest}
                cases.append(cur)
            elif key == "cite":
                cur["cite"] = rest
            elif key == "n":
                cur["n"] = int(rest)
            elif key == "edges":
                cur["edges"] = [tuple(int(x) for x in e.split("-")) for e in rest.split()]
            elif key == "problem":
                kind, bound = rest.split()
                cur["mode"] = 0 if kind == "mvc" else 1
                cur["bound"] = int(bound)
            elif key == "rules":
                bits = 0
                for r in rest.split(","):
                    bits |= {"deg1": 1, "deg2tri": 2, "high": 4, "none": 0}[r]
                cur["rules"] = bits
            elif key in ("start_deg", "expect_deg"):
                cur[key] = [int(x) for x in rest.split()]
            elif key in ("start_S", "start_m", "expect_S", "expect_m", "expect_pruned"):
                cur[key] = int(rest)
            else:
                raise ValueError(f"unknown field {key!r} in {path}")
    return cases


def load_greedy_cases(path: str | None = None) -> list:
    path = path or os.path.join(GOLDEN, "greedy.txt")
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "case":
                cur = {"name": rest}
                cases.append(cur)
            elif key == "cite":
                cur["cite"] = rest
            elif key == "n":
                cur["n"] = int(rest)
            elif key == "edges":
                cur["edges"] = [tuple(int(x) for x in e.split("-")) for e in rest.split()]
            elif key == "expect_greedy":
                cur["expect_greedy"] = int(rest)
            elif key == "expect_cover":
                cur["expect_cover"] = sorted(int(x) for x in rest.split())
            else:
                raise ValueError(f"unknown field {key!r} in {path}")
    return cases
