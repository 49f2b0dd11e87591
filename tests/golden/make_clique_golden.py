"""Writes tests/golden/planted_clique_mvc.txt: the oracle's minimum cover size for members of the
G(n, 0.05) + planted K_c family (c = round(25 n / 400), seed 0) that the oracle can finish.

Calls only the CPU oracle (oracle/) and the seeded generators; each size runs in its own process:
    python tests/golden/make_clique_golden.py 200 240
"""
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "planted_clique_mvc.txt")


def solve(n):
    import oracle
    from paper_2204_10402_gb300 import graphs as G
    c = round(25 * n / 400)
    g, _ = G.gnp_with_planted_clique(n, 0.05, c, 0)
    t0 = time.time()
    size, cover, st = oracle.mvc(g)
    assert oracle.verify_cover(g, cover) and cover.sum() == size
    return n, c, g.m, size, st["nodes"], round(time.time() - t0, 1)


def main():
    import oracle
    oracle.build()
    sizes = [int(x) for x in sys.argv[1:]] or [200]
    with mp.get_context("spawn").Pool(len(sizes)) as pool:
        rows = pool.map(solve, sizes)
    old = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if not line.startswith("#"):
                old[int(line.split()[0])] = line.strip()
    for r in rows:
        old[r[0]] = " ".join(str(x) for x in r)
    with open(OUT, "w") as f:
        f.write("# Oracle minimum vertex cover sizes of G(n, 0.05) + planted K_c, c = round(25 n / 400), seed 0.\n")
        f.write("# Written by tests/golden/make_clique_golden.py (CPU oracle only).\n")
        f.write("# columns: n c m mvc oracle_nodes oracle_seconds\n")
        for k in sorted(old):
            f.write(old[k] + "\n")


if __name__ == "__main__":
    main()
