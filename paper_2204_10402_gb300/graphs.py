"""Seeded synthetic graph generators shared by the tests, the benchmark and the oracle harness.

This module holds no vertex-cover arithmetic: it only draws random numbers and lays graphs out as
CSR.  Every graph is finite, simple and undirected (Sec. II-A): the CSR lists each edge in both
directions, neighbour lists are sorted, there are no self-loops and no duplicates (Sec. IV-B).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used in counter mode: draw ``i`` of stream ``seed`` is the output of
SplitMix64's mixing function applied to ``seed + (i + 1) * 0x9E3779B97F4A7C15``, which is exactly
the ``i``-th output of a SplitMix64 generator whose state starts at ``seed``.  Counter mode makes
every draw addressable, so whole graphs are generated with vectorised numpy arithmetic.  A draw
becomes a double in [0, 1) from its top 53 bits.

Workload shapes follow the paper's two graph families (Sec. V-A, Table I): dense-ish graphs
(stand-ins for the complemented DIMACS p_hat graphs) are Erdos-Renyi G(n, p); sparse power-law
graphs (stand-ins for the KONECT/SNAP graphs) are Chung-Lu graphs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream that starts at state ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2**-53."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class CSR:
    """An undirected graph in CSR form: ``offsets`` has n+1 entries, ``neighbors`` has 2m."""

    n: int
    offsets: np.ndarray  # int32, n+1
    neighbors: np.ndarray  # int32, offsets[n] = 2m

    @property
    def m(self) -> int:
        return int(self.offsets[-1]) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int32)

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        """Each undirected edge once, as (u, v) with u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.offsets))
        keep = src < self.neighbors
        return src[keep], self.neighbors[keep]


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray) -> CSR:
    """Symmetric CSR from an edge list; drops self-loops and duplicate edges, sorts neighbours."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = np.unique(a * n + b) if a.size else np.zeros(0, dtype=np.int64)
    a, b = key // n, key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=offsets[1:])
    return CSR(n, offsets.astype(np.int32), dst.astype(np.int32))


def _pairs_with_probability(n: int, prob_of_pair, seed: int, draw_offset: int = 0):
    """Includes pair (i, j), i < j, iff its draw < its probability; pairs in lexicographic order.

    Draw ``draw_offset + r`` belongs to the r-th pair of that order.  Returns the selected pairs
    and the number of draws used.
    """
    iu, ju = np.triu_indices(n, k=1)
    count = iu.size
    if count == 0:
        return iu, ju, 0
    u = uniform01(seed, count, draw_offset)
    p = prob_of_pair(iu, ju)
    sel = u < p
    return iu[sel], ju[sel], count


def gnp(n: int, p: float, seed: int, draw_offset: int = 0) -> CSR:
    """Erdos-Renyi G(n, p): each pair i < j is an edge iff its uniform draw is below p."""
    i, j, _ = _pairs_with_probability(n, lambda a, b: p, seed, draw_offset)
    return csr_from_edges(n, i, j)


def chung_lu_weights(n: int, avg_degree: float, exponent: float = 2.5, cap: float = 200.0) -> np.ndarray:
    """Expected-degree weights w_i = (i+1)^(-1/(exponent-1)), scaled to mean ``avg_degree``, then capped.

    The cap is applied after scaling and the weights are not rescaled afterwards, so the realised
    average degree can fall slightly below ``avg_degree``.
    """
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (exponent - 1.0))
    w *= avg_degree / w.mean()
    return np.minimum(w, cap)


def chung_lu(n: int, avg_degree: float, seed: int, exponent: float = 2.5, cap: float = 200.0) -> CSR:
    """Chung-Lu graph: pair i < j is an edge with probability min(1, w_i w_j / sum(w))."""
    w = chung_lu_weights(n, avg_degree, exponent, cap)
    total = w.sum()
    i, j, _ = _pairs_with_probability(n, lambda a, b: np.minimum(1.0, w[a] * w[b] / total), seed)
    return csr_from_edges(n, i, j)


def random_subset(n: int, size: int, seed: int, draw_offset: int = 0) -> np.ndarray:
    """A ``size``-subset of range(n): the first ``size`` positions of a partial Fisher-Yates shuffle."""
    perm = np.arange(n, dtype=np.int64)
    u = uniform01(seed, size, draw_offset)
    for i in range(size):
        j = i + min(int(u[i] * (n - i)), n - i - 1)
        perm[i], perm[j] = perm[j], perm[i]
    return np.sort(perm[:size])


def gnp_with_planted_clique(n: int, p: float, clique: int, seed: int) -> tuple[CSR, np.ndarray]:
    """G(n, p) united with a clique on a seeded random ``clique``-subset of the vertices.

    The G(n, p) pairs use draws 0 .. n(n-1)/2 - 1 of the stream; the subset uses the draws after.
    """
    iu, ju, used = _pairs_with_probability(n, lambda a, b: p, seed)
    members = random_subset(n, clique, seed, draw_offset=used)
    ci, cj = np.triu_indices(clique, k=1)
    u = np.concatenate([iu, members[ci]])
    v = np.concatenate([ju, members[cj]])
    return csr_from_edges(n, u, v), members


# ---------------------------------------------------------------------------------------------
# Batches of independent graphs (many small G(n, p) graphs of uneven size)
# ---------------------------------------------------------------------------------------------

@dataclass
class PackedBatch:
    """G graphs packed back to back: graph g owns vertices vtx[g]..vtx[g+1]-1 (renumbered from 0
    inside the graph) and CSR entries edge[g]..edge[g+1]-1 of ``neighbors``; ``offsets`` holds each
    graph's own n_g+1 offsets back to back (Σ(n_g+1) entries), local to the graph."""

    graphs: list
    vtx: np.ndarray  # int32, G+1: prefix sums of n_g
    edge: np.ndarray  # int32, G+1: prefix sums of 2 m_g
    offsets: np.ndarray  # int32, Σ (n_g + 1)
    neighbors: np.ndarray  # int32, Σ 2 m_g


def pack(graphs: list) -> PackedBatch:
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    es = np.array([int(g.offsets[-1]) for g in graphs], dtype=np.int64)
    vtx = np.zeros(len(graphs) + 1, dtype=np.int64)
    edge = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=vtx[1:])
    np.cumsum(es, out=edge[1:])
    offsets = np.concatenate([g.offsets for g in graphs]) if graphs else np.zeros(0, np.int32)
    nbrs = np.concatenate([g.neighbors for g in graphs]) if graphs else np.zeros(0, np.int32)
    return PackedBatch(graphs, vtx.astype(np.int32), edge.astype(np.int32),
                       offsets.astype(np.int32), nbrs.astype(np.int32))


def batch_gnp_params(g: int, n_lo: int = 20, n_hi: int = 120, p_lo: float = 0.05, p_hi: float = 0.30):
    """Graph g draws n ~ U{n_lo..n_hi} (draw 0) and p ~ U[p_lo, p_hi) (draw 1) from stream g."""
    u = uniform01(g, 2)
    n = n_lo + min(int(u[0] * (n_hi - n_lo + 1)), n_hi - n_lo)
    p = p_lo + u[1] * (p_hi - p_lo)
    return n, p


def batch_gnp(num_graphs: int, first_seed: int = 0, **kw) -> PackedBatch:
    """``num_graphs`` G(n, p) graphs; graph g uses stream first_seed+g, its pairs from draw 2 on."""
    graphs = []
    for g in range(num_graphs):
        s = first_seed + g
        n, p = batch_gnp_params(s, **kw)
        graphs.append(gnp(n, p, s, draw_offset=2))
    return pack(graphs)


# ---------------------------------------------------------------------------------------------
# Served request stream (Poisson arrivals, mixed kinds and sizes)
# ---------------------------------------------------------------------------------------------

@dataclass
class Request:
    arrival_s: float
    kind: int  # 0 = MVC, 1 = PVC
    family: int  # 0 = G(n, p), 1 = Chung-Lu
    n: int
    avg_degree: float
    k_offset: int  # PVC: k = MVC + k_offset, k_offset in {-1, 0}
    seed: int


def request_stream(rate_hz: float, duration_s: float, seed: int = 0, n_lo: int = 50, n_hi: int = 3000,
                   pvc_frac: float = 0.7, deg_lo: float = 4.0, deg_hi: float = 10.0,
                   max_requests: int | None = None) -> list:
    """Poisson arrivals at ``rate_hz`` over ``duration_s``.  Request r uses six draws of stream
    ``seed`` (positions 6r .. 6r+5): inter-arrival gap, kind, family, n (log-uniform), average
    degree, PVC k offset.  Its graph is generated from stream ``seed * 2**32 + r + 1``."""
    out = []
    t = 0.0
    r = 0
    ln_lo, ln_hi = math.log(n_lo), math.log(n_hi)
    while True:
        u = uniform01(seed, 6, 6 * r)
        t += -math.log(1.0 - u[0]) / rate_hz
        if t >= duration_s or (max_requests is not None and r >= max_requests):
            break
        kind = 1 if u[1] < pvc_frac else 0
        family = 0 if u[2] < 0.5 else 1
        n = int(math.floor(math.exp(ln_lo + u[3] * (ln_hi - ln_lo))))
        n = max(n_lo, min(n, n_hi))
        d = deg_lo + u[4] * (deg_hi - deg_lo)
        k_off = -1 if u[5] < 0.5 else 0
        out.append(Request(t, kind, family, n, d, k_off, seed * (1 << 32) + r + 1))
        r += 1
    return out


def request_graph(req: Request) -> CSR:
    if req.family == 0:
        return gnp(req.n, min(1.0, req.avg_degree / max(1, req.n - 1)), req.seed)
    return chung_lu(req.n, req.avg_degree, req.seed)


# ---------------------------------------------------------------------------------------------
# Named small graphs with textbook cover sizes (used as fixtures)
# ---------------------------------------------------------------------------------------------

def path(n: int) -> CSR:
    a = np.arange(max(n - 1, 0))
    return csr_from_edges(n, a, a + 1)


def cycle(n: int) -> CSR:
    a = np.arange(n)
    return csr_from_edges(n, a, (a + 1) % n)


def complete(n: int) -> CSR:
    i, j = np.triu_indices(n, k=1)
    return csr_from_edges(n, i, j)


def complete_bipartite(a: int, b: int) -> CSR:
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return csr_from_edges(a + b, i.ravel(), j.ravel())


def star(leaves: int) -> CSR:
    return csr_from_edges(leaves + 1, np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1))


def petersen() -> CSR:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return csr_from_edges(10, e[:, 0], e[:, 1])


def disjoint_union(a: CSR, b: CSR) -> CSR:
    ua, va = a.edges()
    ub, vb = b.edges()
    return csr_from_edges(a.n + b.n, np.concatenate([ua, ub + a.n]), np.concatenate([va, vb + a.n]))


def random_tree_parents(n: int, seed: int) -> np.ndarray:
    """Random recursive tree: vertex i >= 1 hangs below a uniform earlier vertex; parent[0] = -1."""
    parent = np.full(n, -1, dtype=np.int64)
    if n > 1:
        u = uniform01(seed, n - 1)
        i = np.arange(1, n)
        parent[1:] = np.minimum((u * i).astype(np.int64), i - 1)
    return parent


def random_tree(n: int, seed: int) -> CSR:
    parent = random_tree_parents(n, seed)
    i = np.arange(1, n)
    return csr_from_edges(n, parent[1:], i)


def random_bipartite(a: int, b: int, p: float, seed: int) -> CSR:
    """Bipartite graph with sides 0..a-1 and a..a+b-1; each cross pair is an edge iff its draw < p."""
    u = uniform01(seed, a * b).reshape(a, b)
    i, j = np.nonzero(u < p)
    return csr_from_edges(a + b, i, j + a)
