"""Benchmark: batched exact MVC on one GB300 (and weak-scaled replicas on N GPUs).

Workload (one step): 4096 independent Erdos-Renyi graphs, n ~ U{20..120}, p ~ U[0.05, 0.30],
graph g drawn from seed g (plus rank * 4096 under torchrun), packed CSR int32, solved by one
persistent launch of the whole hot path: CSR validation, greedy bound, traversal (reduction rules,
stop check, argmax branch, local stacks + device worklist, termination), results back.

Reported:
  value      solves/s with the packed CSR resident in HBM (CUDA events on the call's stream)
  e2e        solves/s through the C ABI with pinned host buffers (H2D + D2H inside the timing)
  nodes/s, the traversal kernel's roofline, per-request plain launches on the same GPU, the CPU
  oracle on a bounded sample of the same workload, SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "search-tree nodes/sec and solves/sec (p50/p99 latency) vs plain launches; % L2/HBM roofline"
NUM_GRAPHS = 4096
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_GRAPHS = 256  # about 15 s of single-core oracle work
SERVE_WARMUP_S = 3.0     # seconds of the served stream run before its measured legs
SIZE_BINS = ((0, 128), (128, 400), (400, 1000), (1000, 3000))  # n ranges of the served latency breakdown
                                                               # (the first is the server's bit-row class)
PLAIN_SAMPLE_GRAPHS = 512
# Kernels in one replay of the batch plan: worklist init, greedy bound, traversal, answer gather.
KERNELS_PER_STEP = 4
# Records one vc_mvc_batch call copies besides the CSR and the covers (sizes of the C structs,
# checked by tests/test_bench_contract.py): a Problem per graph, the control block, the per-SM
# node counters.
PROBLEM_RECORD_BYTES = 128
CONTROL_BYTES = 1152
SM_COUNTER_BYTES = 1024 * 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--graphs", type=int, default=NUM_GRAPHS)
    ap.add_argument("--no-plain", action="store_true", help="skip the per-request plain-launch leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream leg")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--sweep", default="1000,2000,3000,4000", help="served rates of the sweep (empty: none)")
    ap.add_argument("--sweep-seconds", type=float, default=10.0)
    ap.add_argument("--plain-rate", type=float, default=1000.0, help="rate of the equal-load comparison")
    ap.add_argument("--plain-seconds", type=float, default=15.0)
    ap.add_argument("--burst", type=int, default=20000, help="requests of the server's capacity burst")
    ap.add_argument("--no-configs", action="store_true", help="skip configurations 1-3")
    ap.add_argument("--serve-workers", type=int, default=0,
                    help="CSR-walk workers of the server (0: its default split of the SMs)")
    ap.add_argument("--serve-csr-only", action="store_true", help="serve every request on CSR walks")
    ap.add_argument("--serve-classes", action="store_true", help="serve graphs of <= 128 vertices on bit rows")
    ap.add_argument("--serve-threads", type=int, default=0, help="threads per CSR-walk worker of the server")
    ap.add_argument("--serve-only", action="store_true", help="run only the served-stream leg")
    return ap.parse_args()


def sweep_rates(a) -> tuple:
    return tuple(float(x) for x in a.sweep.split(",") if x.strip())


def serve_config(vc, a):
    """The server's configuration from the command line (None: the library's defaults)."""
    kw = {}
    if a.serve_workers > 0:
        kw["num_workers"] = a.serve_workers
    if a.serve_csr_only:
        kw["bit_rows"] = -1
    if a.serve_classes:
        kw["bit_rows"] = 1
    if a.serve_threads > 0:
        kw["worker_threads"] = a.serve_threads
    return vc.make_config(**kw) if kw else None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int, count: int):
    """Rank r solves its own graphs: streams r*4096 .. r*4096+count-1 (weak scaling, no overlap)."""
    from paper_2204_10402_gb300 import graphs as G
    return G.batch_gnp(count, first_seed=rank * NUM_GRAPHS)


def combine(t_local: float, solves_local: int, device=None):
    """Whole-job figures from every rank's own timing: the slowest rank's time and the sum of
    the solves.  The ranks exchange only these two numbers (no data-path collective)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_local, solves_local
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    n = torch.tensor([solves_local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def e2e_copy_bytes(b, total_n: int) -> tuple[int, int]:
    """Bytes one vc_mvc_batch call with host buffers copies: up, the packed CSR, the problem table
    and the expected neighbour-list lengths; down, the problem table, the control block, the
    per-SM node counters and the cover masks (total_n int32)."""
    G = len(b.vtx) - 1
    h2d = int(b.offsets.nbytes + b.neighbors.nbytes) + G * (PROBLEM_RECORD_BYTES + 8)
    d2h = G * PROBLEM_RECORD_BYTES + CONTROL_BYTES + SM_COUNTER_BYTES + 4 * int(total_n)
    return h2d, d2h


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The files that define the profiled traversal kernel (its code, layout and launch).
TRAVERSAL_SOURCES = ("vc_internal.h", "vc_device.cuh", "vc_rows.cuh", "vc_kernels.cuh", "vc_launch.h",
                     "vc_launch_impl.cuh", "vc_kern_w16_rows.cu", "vc_kern_w32_rows.cu")


def code_only(text: str) -> str:
    """C/C++/CUDA source without its comments, indentation or blank lines (no string literal in
    the traversal sources contains a comment marker)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.strip() for line in text.splitlines() if line.strip())


def traversal_source_hash(csrc: str | None = None) -> str:
    """Hash of the traversal kernel's code: a change of code anywhere in TRAVERSAL_SOURCES changes
    it, a change of comments or layout does not."""
    import hashlib
    csrc = csrc or os.path.join(ROOT, "paper_2204_10402_gb300", "csrc")
    h = hashlib.sha256()
    for f in TRAVERSAL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_per_node(key: str = "dram_bytes_per_tree_node"):
    """A per-tree-node figure of the traversal kernel (DRAM bytes, warp instructions) from the
    committed ncu summary, or None when the kernel's code changed since that capture (the
    summary records its hash)."""
    path = os.path.join(ROOT, "profiles", "traverse_kernel_batch_gnp.md")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line and line.split(":")[0] in ("kernel_source_hash", key):
            k, v = line.split(":", 1)
            rec[k] = v.strip()
    if rec.get("kernel_source_hash") != traversal_source_hash() or key not in rec:
        return None
    return float(rec[key])


def l2_copy_peak(vc, dev) -> float:
    """GB/s (read + write bytes) of the library's L2 copy probe: 16 MiB copied onto another 16 MiB
    64 times in one launch (working set 32 MiB, well inside each die's L2 half), best of 5."""
    import torch
    a = torch.ones(4 << 20, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    stream = torch.cuda.current_stream(dev)
    passes = 64
    vc.l2_copy_probe(b, a, 4, stream)
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vc.l2_copy_probe(b, a, passes, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * a.numel() * 4 * passes / (best * 1e-3) / 1e9


# ------------------------------------------------------------------------------------------------
# CPU oracle legs (test infrastructure, timed as the reported baseline)
# ------------------------------------------------------------------------------------------------

def _oracle_sizes(args):
    import oracle
    from paper_2204_10402_gb300 import graphs as G
    seeds = args
    out = []
    for s in seeds:
        n, p = G.batch_gnp_params(s)
        out.append(oracle.mvc(G.gnp(n, p, s, draw_offset=2))[0])
    return out


def oracle_solves(seeds: list, cores: int):
    """Solves the given batch graphs with the oracle on `cores` processes; returns seconds."""
    import oracle
    oracle.build()
    if cores <= 1:
        t0 = time.perf_counter()
        _oracle_sizes(seeds)
        return time.perf_counter() - t0
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    chunks = [seeds[i::cores] for i in range(cores)]
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_sizes, [[0]] * cores)  # warm the workers (import + load) before timing
        t0 = time.perf_counter()
        pool.map(_oracle_sizes, chunks)
        return time.perf_counter() - t0


def workload_name(graphs: int) -> str:
    """The benchmark workload, named the same way by both arms."""
    return (f"batched MVC, {graphs} G(n,p) graphs per GPU, n~U{{20..120}}, p~U[0.05,0.30], "
            "seed = graph index (+ rank*4096), packed CSR int32, one CUDA-graph launch per step")


def run_reference(a):
    """The oracle as the reference arm: each step solves a bounded sample of the same workload
    (24 graphs, cycling through the 4096) on all host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = min(os.cpu_count() or 1, 16)
    per_step = 24
    for w in range(a.warmup):
        oracle_solves([(w * per_step + i) % NUM_GRAPHS for i in range(per_step)], cores)
    t = 0.0
    done = 0
    for s in range(a.steps):
        base = (a.warmup + s) * per_step
        t += oracle_solves([(base + i) % NUM_GRAPHS for i in range(per_step)], cores)
        done += per_step
    v = done / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * t / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(NUM_GRAPHS), "graphs_per_step": NUM_GRAPHS,
                   "parallelism": "replicas x1", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"a bounded sample of the workload: {per_step} of its graphs per step, "
                                   "cycling through the batch, on all host cores (up to 16)"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU leg
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to $VC_CLOCKS_DIR (default: the system temp dir); the JSON line summarises them
        import tempfile
        self.path = os.path.join(os.environ.get("VC_CLOCKS_DIR", tempfile.gettempdir()), f"vc_clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2204_10402_gb300 as vc
    from paper_2204_10402_gb300 import build

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    vc.load()

    b = workload(rank, a.graphs)
    off_d = torch.from_numpy(b.offsets).to(dev)
    nbr_d = torch.from_numpy(b.neighbors).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    total_n = int(b.vtx[-1])

    # The batch as one CUDA graph (built once, outside the timed region): each step replays the
    # whole launch sequence and reads the answers back.
    plan = vc.BatchPlan(b.vtx, b.edge, off_d, nbr_d)

    def step_device():
        plan.launch(stream)
        sizes, _, st = plan.results(stream)
        return sizes, st

    for _ in range(a.warmup):
        step_device()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    # ---- timed region: K steps, inputs resident in HBM, L2 flushed between steps ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    kernel_ms, stats = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(a.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            sizes, st = step_device()
            ev[i][1].record(stream)
            kernel_ms.append(st["kernel_ms"])
            stats.append(st)
        torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    answered_ms = plan.completion_ms(stream)  # per graph of the last timed step (after the timing)
    want = None
    gold = os.path.join(ROOT, "tests", "golden", "batch4096_mvc.txt")
    if rank == 0 and a.graphs == NUM_GRAPHS and os.path.exists(gold):
        want = [int(l.split()[3]) for l in open(gold) if not l.startswith("#")]
    wrong = None if want is None else int(sum(int(x) != y for x, y in zip(sizes, want)))
    # The same batch through the synchronous vc_mvc_batch call (device-resident CSR, no graph).
    call_ms = []
    for i in range(min(a.steps, 3)):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vc.mvc_batch(b.vtx, b.edge, off_d, nbr_d, stream=stream, want_covers=False)
        call_ms.append(1000 * (time.perf_counter() - t0))
    t_local = sum(step_ms) / 1000.0
    t_max, solves = combine(t_local, a.graphs * a.steps, dev)
    if world > 1:
        dist.barrier()
    value = solves / t_max
    nodes = sum(s["nodes_visited"] for s in stats)

    # ---- e2e: the same call with pinned host buffers (H2D + D2H inside the timing) ----
    off_h = torch.from_numpy(b.offsets).pin_memory()
    nbr_h = torch.from_numpy(b.neighbors).pin_memory()
    e2e_ms = []
    for i in range(a.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sizes_h, covers_h, st_h = vc.mvc_batch(b.vtx, b.edge, off_h.numpy(), nbr_h.numpy(), stream=stream)
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    G = a.graphs
    h2d, d2h = e2e_copy_bytes(b, total_n)
    e2e_value = solves / world / (sum(e2e_ms) / 1000.0) * world if e2e_ms else None

    out = None
    if rank == 0:
        # ---- roofline of the traversal kernel: algorithmic bytes / its event-timed duration ----
        hbm, peak_kind = peaks()
        alg_bytes = [s["entry_bytes_moved"] + 4 * s["csr_words"] for s in stats]
        ach = [bb / (km * 1e-3) / 1e9 for bb, km in zip(alg_bytes, kernel_ms) if km > 0]
        achieved = statistics.mean(ach) if ach else 0.0
        per_node = measured_per_node("dram_bytes_per_tree_node")
        inst_per_node = measured_per_node("warp_instructions_per_tree_node")
        nodes_per_launch = statistics.mean(s["nodes_visited"] for s in stats)
        l2_peak = l2_copy_peak(vc, dev)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm,
                    "traffic": per_node * nodes_per_launch if per_node is not None else None,
                    "traffic_note": "ncu dram bytes per tree node of the full 4096-graph launch (1 pass) x nodes of this launch",
                    "peak_kind": peak_kind, "kernel": "traverse_kernel",
                    "kernel_ms_mean": statistics.mean(kernel_ms),
                    "alg_bytes_per_launch": statistics.mean(alg_bytes),
                    "l2": {"peak_probe_gbs": l2_peak, "frac": achieved / l2_peak,
                           "probe": "vc_l2_copy_probe: 16 MiB onto 16 MiB x 64 passes in one launch, .cg loads/stores, read+write bytes"}}
        if inst_per_node is not None:
            # What actually bounds the traversal: warp-instruction issue.  Instructions per node
            # from the ncu capture x nodes of this launch / its event time, against one warp
            # instruction per scheduler per cycle (4 per SM) at the SM clock sampled in the run.
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            mhz = clk.summary().get("sm_mhz") or 0.0
            ginst = inst_per_node * nodes_per_launch / (statistics.mean(kernel_ms) * 1e-3) / 1e9
            peak_ginst = sms * 4 * mhz / 1e3
            roofline["issue"] = {"achieved": ginst, "peak": peak_ginst, "unit": "G warp-inst/s",
                                 "frac": ginst / peak_ginst if peak_ginst else None,
                                 "note": "ncu warp instructions per tree node (full 4096-graph launch) x nodes / kernel time; "
                                         "peak = SMs x 4 schedulers x sampled SM clock"}
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000 * t_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name(G),
                       "graphs_per_step": G, "sum_n": total_n, "sum_2m": int(b.edge[-1]),
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"replicas x{world}",
                       "variant": {"width": stats[0]["width"], "worker_threads": stats[0]["worker_threads"],
                                   "workers": stats[0]["workers"]}},
            "nodes_per_s": nodes * world / t_max,
            "load_balance": load_balance(vc),
            "wrong_answers_vs_oracle": wrong,
            "batch_call_solves_per_s": a.graphs / (statistics.mean(call_ms) / 1000.0),
            "nodes_per_step": nodes / a.steps,
            "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99)),
                           "note": "a caller gets every graph's answer with the step (p50 / p99 of the step time)",
                           "per_graph_answered_ms": {
                               "p50": float(np.percentile(answered_ms, 50)), "p99": float(np.percentile(answered_ms, 99)),
                               "max": float(answered_ms.max()) if answered_ms.size else None,
                               "note": "when each graph of the last timed step was answered (its greedy bound, or the "
                                       "end of its own search), from the step's greedy pass"}},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": KERNELS_PER_STEP * a.steps,
            "roofline": roofline,
        }
        if not a.no_plain:
            line["vs_plain_launches"] = plain_launches(vc, b, dev, stream, value)
        clocks = clk.summary()
        line["clocks"] = clocks
        if not a.no_serve and world == 1:
            line["serving"] = serving_leg(vc, a.serve_rate, a.serve_seconds, sweep_rates(a), a.sweep_seconds,
                                          a.plain_rate, a.plain_seconds, a.burst, config=serve_config(vc, a))
        if not a.no_configs and world == 1:
            line["configs"] = configs_leg(vc, dev, local, with_oracle=not a.no_cpu)
        if not a.no_cpu and world == 1:
            seeds = list(range(min(CPU_SAMPLE_GRAPHS, G)))
            secs = oracle_solves(seeds, 1)
            line["cpu_baseline"] = {"value": len(seeds) / secs, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": f"first {len(seeds)} graphs of the batch, one core, {secs:.1f} s"}
        out = line
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def load_balance(vc):
    """Sec. V-C load measure for the last traversal: tree nodes per SM over the mean."""
    per_sm = vc.last_sm_nodes().astype(np.float64)
    per_sm = per_sm[per_sm > 0] if per_sm.any() else per_sm
    if per_sm.size == 0:
        return None
    mean = per_sm.mean()
    return {"sms": int(per_sm.size), "min_over_mean": float(per_sm.min() / mean),
            "max_over_mean": float(per_sm.max() / mean)}


def load_serve_pool():
    """Oracle-solved request graphs of the served workload (tests/golden/serve_pool.txt)."""
    from paper_2204_10402_gb300 import graphs as G
    path = os.path.join(ROOT, "tests", "golden", "serve_pool.txt")
    pool, total = [], 0
    for line in open(path):
        if line.startswith("#"):
            continue
        seed, fam, n, d, m, mvc, nodes = line.split()
        total += 1
        if int(mvc) < 0:
            continue
        pool.append(dict(req=G.Request(0.0, 0, int(fam), int(n), float(d), 0, int(seed)), mvc=int(mvc)))
    return pool, total


def served_requests(rate_hz: float, duration_s: float, pool: list):
    """The seeded Poisson stream (seed 0): request i picks a pool graph with draw i of stream 2^40,
    is PVC with probability 0.7 (k = MVC-1 or MVC) else MVC.  Every rate sees the same sequence of
    requests; only the arrival times scale.  Items: (arrival_s, kind, k, pool entry, answer)."""
    from paper_2204_10402_gb300 import graphs as G
    stream = G.request_stream(rate_hz, duration_s, seed=0)
    pick = G.uniform01(1 << 40, max(len(stream), 1))
    reqs = []
    for r, u in zip(stream, pick):
        e = pool[min(int(u * len(pool)), len(pool) - 1)]
        k = e["mvc"] + r.k_offset if r.kind == 1 else 0
        want = e["mvc"] if r.kind == 0 else int(k >= e["mvc"])
        reqs.append((r.arrival_s, r.kind, k, e, want))
    return reqs


def _percentiles(lat_ms) -> dict:
    lat = np.asarray(lat_ms, dtype=np.float64)
    if lat.size == 0:
        return {"p50": None, "p99": None, "p999": None}
    return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
            "p999": float(np.percentile(lat, 99.9))}


def run_served(srv, reqs, graphs, burst: bool = False) -> dict:
    """Open loop: each request is submitted at its scheduled arrival (all at once with burst) and its
    latency is the completion the host sees minus that arrival.  Records are released as read."""
    st0 = srv.stats()
    ids = []
    gc.disable()  # a collector pause would delay submissions and show up as request latency
    try:
        t0 = time.monotonic_ns() + 2_000_000
        for arr, kind, k, e, want in reqs:
            due = t0 if burst else t0 + int(arr * 1e9)
            while time.monotonic_ns() < due:
                pass
            g = graphs[e["req"].seed]
            ids.append(srv.submit(g.offsets, g.neighbors, kind, k))
        srv.drain(timeout_ms=900000)
    finally:
        gc.enable()
    infos = [srv.poll(i, release=True) for i in ids]
    st1 = srv.stats()
    due = [t0 if burst else t0 + int(r[0] * 1e9) for r in reqs]
    lat = [(x["done_ns"] - d) / 1e6 for x, d in zip(infos, due)]
    lag = [(x["submit_ns"] - d) / 1e6 for x, d in zip(infos, due)]
    wrong = sum(1 for x, r in zip(infos, reqs) if x["answer"] != r[4] or x["status"] != 0)
    span = (max(x["done_ns"] for x in infos) - t0) / 1e9 if infos else 0.0
    sizes = [r[3]["req"].n for r in reqs]
    bins = {}
    for lo, hi in SIZE_BINS:
        sel = [x for x, n in zip(lat, sizes) if lo < n <= hi]
        bins[f"{lo + 1}-{hi}"] = {"requests": len(sel), **_percentiles(sel)}
    return {"requests": len(reqs), "wrong_answers": wrong,
            "solves_per_s": len(reqs) / span if span > 0 else None,
            "latency_ms": _percentiles(lat),
            "submit_lag_ms": _percentiles(lag),
            "latency_ms_by_n": bins,
            "launches": st1["launches"] - st0["launches"], "nodes_visited": st1["nodes_visited"] - st0["nodes_visited"],
            "records_held_after": st1["records"]}


def run_plain_open_loop(vc, reqs, dev_graphs) -> dict:
    """Per-request plain launches, open loop: one host thread makes one synchronous vc_mvc / vc_pvc
    call per request (device-resident CSR), starting at the request's arrival or, if the previous
    call is still running, when it returns; latency = return - arrival."""
    lat, wrong, busy = [], 0, 0.0
    gc.disable()  # as in run_served: no collector pause inside the open loop
    try:
        t0 = time.monotonic_ns() + 2_000_000
        for arr, kind, k, e, want in reqs:
            due = t0 + int(arr * 1e9)
            while time.monotonic_ns() < due:
                pass
            off, nbr = dev_graphs[e["req"].seed]
            s = time.monotonic_ns()
            a = vc.mvc(off, nbr, want_cover=False) if kind == 0 else vc.pvc(off, nbr, k, want_cover=False)
            done = time.monotonic_ns()
            busy += (done - s) / 1e9
            lat.append((done - due) / 1e6)
            wrong += int(a.value != want)
        span = (time.monotonic_ns() - t0) / 1e9
    finally:
        gc.enable()
    return {"requests": len(reqs), "wrong_answers": wrong, "solves_per_s": len(reqs) / span,
            "latency_ms": _percentiles(lat), "capacity_solves_per_s": len(reqs) / busy if busy else None}


def serving_leg(vc, rate_hz: float, duration_s: float, sweep_rates=(), sweep_s: float = 10.0,
                plain_rate: float = 1000.0, plain_s: float = 15.0, burst: int = 20000, budget_gib: int = 64,
                config=None):
    """The served workload: the stream at rate_hz for duration_s, a rate sweep, the server's
    capacity under a burst, and plain launches against the server at one rate both sustain."""
    import torch
    from paper_2204_10402_gb300 import graphs as G
    pool, total = load_serve_pool()
    graphs = {}
    for e in pool:
        graphs[e["req"].seed] = G.request_graph(e["req"])
    max_n = max(g.n for g in graphs.values())
    srv = vc.Server(max_n=max_n, budget_bytes=budget_gib << 30, config=config)
    # Warm-up: a burst (module load, first launches), then 3 s of the stream itself.  A process's
    # first seconds with two size classes running side by side have shown one stall of 15-55 ms
    # (the server thread waiting in the CUDA driver); the warm-up keeps it out of the measurement.
    run_served(srv, served_requests(2000.0, 0.05, pool), graphs, burst=True)
    run_served(srv, served_requests(2000.0, SERVE_WARMUP_S, pool), graphs)
    main = run_served(srv, served_requests(rate_hz, duration_s, pool), graphs)
    out = {
        "workload": f"Poisson {rate_hz:g} req/s for {duration_s:g} s, 70% PVC (k = MVC-1 or MVC) / 30% MVC, "
                    f"graphs from a pool of {len(pool)} oracle-solved requests "
                    f"({total - len(pool)} of {total} candidates rejected over a 50K-node oracle cap)",
        **main,
    }
    st = srv.stats()
    out["server"] = {k: st[k] for k in ("epochs", "workers", "worker_threads", "classes", "small_max_n",
                                         "small_workers")}
    if sweep_rates:
        out["rate_sweep"] = []
        for r in sweep_rates:
            res = run_served(srv, served_requests(r, sweep_s, pool), graphs)
            out["rate_sweep"].append({"offered_per_s": r, "seconds": sweep_s, **res})
    if burst > 0:
        reqs = served_requests(2000.0, burst / 2000.0 + 1.0, pool)[:burst]
        res = run_served(srv, reqs, graphs, burst=True)
        out["capacity_burst"] = {"requests": res["requests"], "solves_per_s": res["solves_per_s"],
                                 "wrong_answers": res["wrong_answers"],
                                 "note": "all requests submitted at once; completions per second of the span"}
    if plain_rate > 0 and plain_s > 0:
        reqs = served_requests(plain_rate, plain_s, pool)
        served = run_served(srv, reqs, graphs)
        dev_graphs = {key: (torch.from_numpy(g.offsets).cuda(),
                            torch.from_numpy(g.neighbors if g.neighbors.size else np.zeros(1, np.int32)).cuda())
                      for key, g in graphs.items()}
        for key in list(dev_graphs)[:16]:  # warm-up of the plain path
            vc.mvc(*dev_graphs[key], want_cover=False)
        torch.cuda.synchronize()
        plain = run_plain_open_loop(vc, reqs, dev_graphs)
        out["equal_load"] = {"offered_per_s": plain_rate, "seconds": plain_s, "served": served,
                             "plain_launches": plain,
                             "note": "the same requests and arrival times through the server and through one "
                                     "synchronous vc_mvc / vc_pvc call each (device-resident CSR)"}
    srv.close()
    return out


def configs_leg(vc, dev, local: int, with_oracle: bool = True) -> dict:
    """Configurations 1-3 of the workload set, each timed on the GPU (CUDA-synchronous calls through
    the C ABI, device-resident CSR) with its answer checked, beside the single-core oracle."""
    import torch

    import oracle
    from paper_2204_10402_gb300 import graphs as G
    oracle.build()

    def dev_csr(g):
        return (torch.from_numpy(g.offsets).to(dev),
                torch.from_numpy(g.neighbors if g.neighbors.size else np.zeros(1, np.int32)).to(dev))

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            t = time.perf_counter()
            r = fn()
            ms.append(1000 * (time.perf_counter() - t))
        return r, ms

    def oracle_ms(fn, reps):
        ms = []
        for _ in range(reps):
            t = time.perf_counter()
            r = fn()
            ms.append(1000 * (time.perf_counter() - t))
        return r, statistics.median(ms)

    out = {}
    with ClockSampler(local) as clk:
        # 1: MVC of G(60, 0.10), seed 0, with a verified cover; a single request.
        g1 = G.gnp(60, 0.10, 0)
        want1 = oracle.mvc(g1)[0]
        off, nbr = dev_csr(g1)
        a1, ms1 = timed(lambda: vc.mvc(off, nbr), 200)
        cover = a1.cover.cpu().numpy().astype(bool)
        _, ms1h = timed(lambda: vc.mvc(g1.offsets, g1.neighbors), 50)
        out["config1"] = {"workload": "MVC of G(60, 0.10), seed 0, one request", "mvc": a1.value,
                          "correct": a1.value == want1 and int(cover.sum()) == a1.value and oracle.verify_cover(g1, cover),
                          "latency_ms": {"p50": statistics.median(ms1), "p99": float(np.percentile(ms1, 99))},
                          "latency_host_arrays_ms_p50": statistics.median(ms1h), "nodes": a1.stats["nodes_visited"]}
        # 2: PVC on Chung-Lu n=2000 (avg degree 6, exponent 2.5, cap 200), seed 0, k = MVC and MVC-1.
        g2 = G.chung_lu(2000, 6.0, 0)
        mvc2 = oracle.mvc(g2)[0]
        off, nbr = dev_csr(g2)
        c2 = {"workload": "PVC of Chung-Lu n=2000 (average degree 6, exponent 2.5, cap 200), seed 0", "mvc": mvc2}
        for name, k, want in (("k_mvc", mvc2, 1), ("k_mvc_minus_1", mvc2 - 1, 0)):
            a2, ms2 = timed(lambda: vc.pvc(off, nbr, k), 50)
            c2[name] = {"k": k, "found": a2.value, "correct": a2.value == want,
                        "latency_ms": {"p50": statistics.median(ms2), "p99": float(np.percentile(ms2, 99))},
                        "nodes": a2.stats["nodes_visited"]}
        out["config2"] = c2
        # 3: the largest member of the G(n, 0.05) + planted K_{25n/400} family that finishes: n = 200
        # (n = 400 is intractable for this method), 32- and 16-bit degree arrays.
        gold = {int(l.split()[0]): l.split() for l in open(os.path.join(ROOT, "tests", "golden", "planted_clique_mvc.txt"))
                if not l.startswith("#")}
        g3, _ = G.gnp_with_planted_clique(200, 0.05, 12, 0)
        off, nbr = dev_csr(g3)
        c3 = {"workload": "MVC of G(200, 0.05) + planted K_12, seed 0 (the n = 400 member is intractable)",
              "mvc_oracle_stored": int(gold[200][3])}
        for width in (32, 16):
            cfg = vc.make_config(width=width)
            a3, ms3 = timed(lambda: vc.mvc(off, nbr, config=cfg, want_cover=False), 2)
            c3[f"int{width}"] = {"mvc": a3.value, "correct": a3.value == int(gold[200][3]),
                                 "ms": min(ms3), "kernel_ms": a3.stats["kernel_ms"], "nodes": a3.stats["nodes_visited"],
                                 "nodes_per_s": a3.stats["nodes_visited"] / (a3.stats["kernel_ms"] * 1e-3)}
        out["config3"] = c3
    out["clocks"] = clk.summary()
    if with_oracle:
        _, o1 = oracle_ms(lambda: oracle.mvc(g1), 5)
        out["config1"]["oracle_1core_ms"] = o1
        _, o2 = oracle_ms(lambda: oracle.pvc(g2, mvc2 - 1), 5)
        out["config2"]["oracle_1core_ms_k_mvc_minus_1"] = o2
        g160, _ = G.gnp_with_planted_clique(160, 0.05, 10, 0)
        r160, o3 = oracle_ms(lambda: oracle.mvc(g160), 1)
        out["config3"]["oracle_1core"] = {
            "n160_ms": o3, "n160_nodes": r160[2]["nodes"],
            "n200_s_stored": float(gold[200][5]), "n200_nodes_stored": int(gold[200][4]),
            "note": "n = 160 timed in this run; n = 200 from tests/golden/planted_clique_mvc.txt (another host)"}
    return out


def plain_launches(vc, b, dev, stream, batched_value):
    """Per-request plain launches: one vc_mvc call per graph (device-resident CSR), same GPU."""
    import torch
    cnt = min(PLAIN_SAMPLE_GRAPHS, len(b.graphs))
    offs = [torch.from_numpy(g.offsets).to(dev) for g in b.graphs[:cnt]]
    nbrs = [torch.from_numpy(g.neighbors if g.neighbors.size else np.zeros(1, np.int32)).to(dev)
            for g in b.graphs[:cnt]]
    for i in range(min(8, cnt)):
        vc.mvc(offs[i], nbrs[i], stream=stream, want_cover=False)
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    for i in range(cnt):
        s = time.perf_counter()
        vc.mvc(offs[i], nbrs[i], stream=stream, want_cover=False)
        lat.append(1000 * (time.perf_counter() - s))
    total = time.perf_counter() - t0
    plain = cnt / total
    return {"plain_solves_per_s": plain, "batched_over_plain": batched_value / plain,
            "plain_latency_ms": {"p50": statistics.median(lat), "p99": float(np.percentile(lat, 99))},
            "sample": f"first {cnt} graphs, one synchronous vc_mvc call each"}


def main():
    a = parse()
    if a.serve_only:
        import paper_2204_10402_gb300 as vc
        from paper_2204_10402_gb300 import build
        build.build()
        vc.load()
        print(json.dumps(serving_leg(vc, a.serve_rate, a.serve_seconds, sweep_rates(a), a.sweep_seconds,
                                     a.plain_rate, a.plain_seconds, a.burst, config=serve_config(vc, a))), flush=True)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
