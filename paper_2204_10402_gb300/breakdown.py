"""Sec. V-C and V-D instrumentation: where a traversal's time goes, and how its tree nodes spread
over the SMs.

Runs the library built with ``-DVC_TRACE`` (``build.build_variant("trace")``), which adds per-worker
activity timers to the traversal kernel (the product library carries none):

  time breakdown   worker time (%globaltimer) waiting for work, in the reduction rules and stop
                   check, branching (argmax, donate or push, the "v" child), capturing solutions:
                   the categories of the paper's Fig. 6
  cycle breakdown  SM cycles of each worker's first thread per finer activity (rule scans,
                   removals, stack pops, worklist work, ...) and the number of rule passes of
                   each kind
  per-SM load      tree nodes expanded per SM over the mean (Fig. 5)

    python -m paper_2204_10402_gb300.breakdown [--graphs 4096] [--clique 200] [--json]

The process loads the trace library, so it runs in a process of its own.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

# ProfSlot order of the kernels' VC_TRACE cycle slots (csrc/vc_device.cuh).
CYCLE_SLOTS = ("snapshot", "degree_one_scans", "triangle_scans", "high_degree_scans", "removals", "stop_checks",
               "argmax", "donate_or_push", "take_v", "stack_pops", "take_neighbourhood", "acquire", "solutions")
PASS_SLOTS = ("degree_one_passes", "triangle_passes", "high_degree_passes")
TIME_SLOTS = ("waiting_for_work", "reduction_rules_and_stop_check", "branching", "solutions")


def summarise(stats: dict, sm_nodes: np.ndarray) -> dict:
    """Shares of the traced activities in one launch's statistics."""
    cyc = stats["trace_cycles"]
    cycles = dict(zip(CYCLE_SLOTS, cyc[: len(CYCLE_SLOTS)]))
    passes = dict(zip(PASS_SLOTS, cyc[len(CYCLE_SLOTS): len(CYCLE_SLOTS) + len(PASS_SLOTS)]))
    total_cyc = sum(cycles.values())
    nodes = max(stats["nodes_visited"], 1)
    ns = dict(zip(TIME_SLOTS, stats["trace_ns"]))
    total_ns = sum(ns.values())
    busy = sm_nodes[sm_nodes > 0].astype(np.float64)
    return {
        "nodes": stats["nodes_visited"],
        "kernel_ms": stats["kernel_ms"],
        "workers": stats["workers"],
        "worker_threads": stats["worker_threads"],
        "bit_rows": stats["bit_rows"],
        "rule_passes": stats["rule_passes"],
        "time_share": {k: (v / total_ns if total_ns else 0.0) for k, v in ns.items()},
        "worker_ns_total": total_ns,
        "cycle_share": {k: (v / total_cyc if total_cyc else 0.0) for k, v in cycles.items()},
        "cycles_per_node": total_cyc / nodes,
        "cycles_total": total_cyc,
        "passes": passes,
        "passes_per_node": sum(passes.values()) / nodes,
        "sm_load": ({"sms": int(busy.size), "min_over_mean": float(busy.min() / busy.mean()),
                     "max_over_mean": float(busy.max() / busy.mean())} if busy.size else None),
    }


def run(graphs: int, clique: int, lib_path: str | None = None) -> dict:
    import torch

    import paper_2204_10402_gb300 as vc
    from paper_2204_10402_gb300 import build
    from paper_2204_10402_gb300 import graphs as G

    vc.load(lib_path or build.build_variant("trace"))
    out = {}
    if graphs > 0:
        b = G.batch_gnp(graphs)
        off = torch.from_numpy(b.offsets).cuda()
        nbr = torch.from_numpy(b.neighbors).cuda()
        vc.mvc_batch(b.vtx, b.edge, off, nbr, want_covers=False)  # warm-up (module load, workspace)
        sizes, _, st = vc.mvc_batch(b.vtx, b.edge, off, nbr, want_covers=False)
        torch.cuda.synchronize()
        out["batch"] = summarise(st, vc.last_sm_nodes())
        out["batch"]["workload"] = f"{graphs} G(n,p) graphs, n~U{{20..120}}, p~U[0.05,0.30], seed = graph index"
        out["batch"]["sizes"] = [int(x) for x in sizes]
    if clique > 0:
        c = round(25 * clique / 400)
        g, _ = G.gnp_with_planted_clique(clique, 0.05, c, 0)
        off = torch.from_numpy(g.offsets).cuda()
        nbr = torch.from_numpy(g.neighbors).cuda()
        # the default workers (bit rows up to 256 vertices), then CSR walks on the same instance
        for key, cfg in (("clique", None), ("clique_csr", vc.make_config(bit_rows=-1))):
            a = vc.mvc(off, nbr, config=cfg)
            torch.cuda.synchronize()
            out[key] = summarise(a.stats, vc.last_sm_nodes())
            out[key]["workload"] = (f"G({clique}, 0.05) + planted K_{c}, seed 0, one instance"
                                    + (", CSR walks" if cfg is not None else ""))
            out[key]["mvc"] = a.value
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=4096, help="batch size (0: skip the batch)")
    ap.add_argument("--clique", type=int, default=200, help="planted-clique n (0: skip)")
    ap.add_argument("--lib", default=None, help="a trace build of libvc.so (default: build it)")
    a = ap.parse_args(argv)
    res = run(a.graphs, a.clique, a.lib)
    for r in res.values():
        r.pop("sizes", None)
    json.dump(res, sys.stdout, indent=1)
    print()


if __name__ == "__main__":
    main()
