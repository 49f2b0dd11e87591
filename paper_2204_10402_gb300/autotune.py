"""Autotuner: picks the launch configuration per graph-size class by measuring it.

Knobs (all fields of vc_config, include/vc.h):
  worker_threads      threads per worker (the paper's block size, Sec. IV-E / V-A)
  width               16- or 32-bit degree-array entries
  donate_threshold    worklist fill fraction below which branches are donated (Sec. IV-A, V-A)
  worklist_capacity   worklist entries (Sec. V-A)
  stage_csr           shared-memory placement of the current graph: offsets (0), offsets and
                      neighbour lists (1), nothing (-1)
  node_in_global      placement of the current node (Sec. IV-E's two kernel versions): shared
                      memory when it fits (0) or global memory (1)
  bit_rows            adjacency lookups: bit rows for graphs up to 256 vertices where they can
                      run (0), bit rows required (1), CSR walks (-1)

Search: coordinate descent from the library's defaults -- each knob in turn is set to the value
with the lowest measured traversal time while the others stay fixed; two sweeps.  Results are
cached per device and size class in a JSON file ($VC_AUTOTUNE_CACHE, else
~/.cache/vc_gb300/autotune.json) and returned by config_for().
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

SIZE_CLASSES = (64, 128, 256, 512, 1024, 2048, 4096, 1 << 31)

SPACE = {
    "worker_threads": (32, 64, 128, 256),
    "width": (16, 32),
    "donate_threshold": (0.25, 0.5, 1.0),
    "worklist_capacity": (65536, 262144, 524288),
    "stage_csr": (0, 1, -1),
    "node_in_global": (0, 1),
    "bit_rows": (0, 1, -1),
}


def size_class(n_max: int) -> int:
    for c in SIZE_CLASSES:
        if n_max <= c:
            return c
    return SIZE_CLASSES[-1]


def cache_path() -> str:
    p = os.environ.get("VC_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "vc_gb300", "autotune.json")


@dataclass
class Trial:
    config: dict
    ms: float


def coordinate_descent(measure, start: dict | None = None, space: dict | None = None, sweeps: int = 2):
    """Minimises measure(config) -> milliseconds (inf when the config is rejected) one knob at a
    time.  Returns (best config, best ms, trials)."""
    space = space or SPACE
    cur = dict(start or {})
    trials = []
    seen = {}

    def run(cfg):
        key = json.dumps(cfg, sort_keys=True)
        if key not in seen:
            ms = measure(cfg)
            seen[key] = ms
            trials.append(Trial(dict(cfg), ms))
        return seen[key]

    best_ms = run(cur)
    for _ in range(sweeps):
        improved = False
        for knob, values in space.items():
            for v in values:
                cand = dict(cur)
                cand[knob] = v
                ms = run(cand)
                if ms < best_ms:
                    best_ms, cur, improved = ms, cand, True
        if not improved:
            break
    return cur, best_ms, trials


def _device_key() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0).replace(" ", "_")
    except Exception:
        return "unknown"


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(table: dict):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def config_for(n_max: int, kind: str = "batch"):
    """The cached tuned config for this size class (a vc_config), or None if none was tuned."""
    import paper_2204_10402_gb300 as vc
    entry = load_cache().get(_device_key(), {}).get(f"{kind}:{size_class(n_max)}")
    return vc.make_config(**entry["config"]) if entry else None


def tune_batch(vtx, edge, offsets, neighbors, repeats: int = 2, sweeps: int = 2, space: dict | None = None,
               save: bool = True):
    """Tunes the batched launch on a sample batch (host arrays or CUDA tensors) and caches the
    result under the batch's size class.  Returns (config dict, ms, trials)."""
    import numpy as np

    import paper_2204_10402_gb300 as vc
    n_max = int(np.max(np.diff(np.asarray(vtx)))) if len(vtx) > 1 else 0
    reference = None

    def measure(cfg):
        nonlocal reference
        try:
            best = float("inf")
            for _ in range(repeats):
                sizes, _, st = vc.mvc_batch(vtx, edge, offsets, neighbors, config=vc.make_config(**cfg),
                                            want_covers=False)
                best = min(best, st["kernel_ms"])
            sizes = [int(x) for x in sizes]
            if reference is None:
                reference = sizes
            elif sizes != reference:  # every configuration must give the same answers
                raise RuntimeError(f"config {cfg} changed the answers")
            return best
        except vc.VCError:
            return float("inf")

    cfg, ms, trials = coordinate_descent(measure, {}, space, sweeps)
    if save:
        table = load_cache()
        table.setdefault(_device_key(), {})[f"batch:{size_class(n_max)}"] = {"config": cfg, "ms": ms}
        save_cache(table)
    return cfg, ms, trials
