"""Writes tests/golden/serve_pool.txt: candidate request graphs of the served workload (G(n,p) or
Chung-Lu with exponent 2.5, average degree ~U[4,10], n log-uniform in [50, 3000]), each solved by
the CPU oracle under a node cap; graphs over the cap are kept with mvc = -1 (rejected).

Candidate c uses the request parameters of draw c of request_stream(seed=0) and its own graph
stream.  Calls only the CPU oracle (oracle/) and the seeded generators:
    python tests/golden/make_serve_pool.py [count] [node_cap] [processes]
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serve_pool.txt")


def solve(args):
    import oracle
    from paper_2204_10402_gb300 import graphs as G
    req, cap = args
    g = G.request_graph(req)
    try:
        size, cover, st = oracle.mvc(g, max_nodes=cap)
        assert oracle.verify_cover(g, cover) and cover.sum() == size
        nodes = st["nodes"]
    except oracle.OracleLimit:
        size, nodes = -1, cap
    return req.seed, req.family, req.n, f"{req.avg_degree:.6f}", g.m, size, nodes


def main():
    import oracle
    from paper_2204_10402_gb300 import graphs as G
    oracle.build()
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    cap = int(sys.argv[2]) if len(sys.argv) > 2 else 50000
    procs = int(sys.argv[3]) if len(sys.argv) > 3 else (os.cpu_count() or 1)
    reqs = G.request_stream(1e9, 1e9, seed=0, max_requests=count)
    with mp.get_context("spawn").Pool(procs) as pool:
        rows = pool.map(solve, [(r, cap) for r in reqs], chunksize=1)
    with open(OUT, "w") as f:
        f.write("# Served-workload request graphs solved by the CPU oracle (mvc = -1: over the node cap).\n")
        f.write(f"# Written by tests/golden/make_serve_pool.py {count} {cap} (CPU oracle only).\n")
        f.write("# columns: graph_seed family(0=gnp,1=chung_lu) n avg_degree m mvc oracle_nodes\n")
        for r in rows:
            f.write(" ".join(str(x) for x in r) + "\n")


if __name__ == "__main__":
    main()
