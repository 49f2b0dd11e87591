"""Writes tests/golden/batch4096_mvc.txt: the oracle's minimum cover size for every graph of the
4096-graph G(n, p) batch (graph g: stream g, n ~ U{20..120}, p ~ U[0.05, 0.30]).

Calls only the CPU oracle (oracle/) and the seeded generators; run with
    python tests/golden/make_batch_golden.py [processes]
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch4096_mvc.txt")


def solve(g_index):
    import oracle
    from paper_2204_10402_gb300 import graphs as G
    n, p = G.batch_gnp_params(g_index)
    g = G.gnp(n, p, g_index, draw_offset=2)
    size, cover, st = oracle.mvc(g)
    assert oracle.verify_cover(g, cover) and cover.sum() == size
    return g_index, n, g.m, size, st["nodes"]


def main():
    import oracle
    oracle.build()
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        rows = sorted(pool.map(solve, range(4096), chunksize=8))
    with open(OUT, "w") as f:
        f.write("# Oracle minimum vertex cover sizes of the 4096-graph G(n,p) batch.\n")
        f.write("# Written by tests/golden/make_batch_golden.py (CPU oracle only).\n")
        f.write("# columns: graph n m mvc oracle_nodes\n")
        for r in rows:
            f.write(" ".join(str(x) for x in r) + "\n")


if __name__ == "__main__":
    main()
