"""The VC_TRACE build (Sec. V-C / V-D instrumentation) against the oracle and against itself.

The instrumented library is built into a directory of its own and loaded by a child process
(a process loads one build of the library).  Checks:
  - its answers equal the oracle's (stored batch answers; the planted-clique instance solved here,
    on bit rows and on CSR walks)
  - every activity slot that both workloads exercise is non-zero
  - the traced worker time and the traced cycles fit inside the kernel's duration x workers
  - the traced pass counts add up to the rule passes the product counters report
  - per-SM load is reported over busy SMs
"""
import json
import os
import subprocess
import sys

import pytest

import oracle
from paper_2204_10402_gb300 import graphs as G

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BATCH = 256
CLIQUE_N = 120


def sm_max_hz() -> float:
    """The GPU's maximum SM clock from nvidia-smi (GB300: 2070 MHz)."""
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=30).stdout.strip().splitlines()
        return float(out[0]) * 1e6
    except Exception:
        return 2070e6


@pytest.fixture(scope="module")
def traced():
    from paper_2204_10402_gb300 import build
    lib = build.build_variant("trace")
    code = ("import json,sys; from paper_2204_10402_gb300 import breakdown as B; "
            f"json.dump(B.run({BATCH}, {CLIQUE_N}, {lib!r}), sys.stdout)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_trace_build_answers_match_oracle(traced):
    gold = os.path.join(ROOT, "tests", "golden", "batch4096_mvc.txt")
    want = [int(l.split()[3]) for l in open(gold) if not l.startswith("#")][:BATCH]
    assert traced["batch"]["sizes"] == want
    c = round(25 * CLIQUE_N / 400)
    g, _ = G.gnp_with_planted_clique(CLIQUE_N, 0.05, c, 0)
    want = oracle.mvc(g)[0]
    assert traced["clique"]["mvc"] == want and traced["clique_csr"]["mvc"] == want
    assert traced["clique"]["bit_rows"] == 4 and traced["clique_csr"]["bit_rows"] == 0


@pytest.mark.parametrize("which", ["batch", "clique", "clique_csr"])
def test_trace_slots_consistent(traced, which):
    r = traced[which]
    assert r["nodes"] > 0 and r["kernel_ms"] > 0
    # Every activity of a branching search shows up.  (Stack pops are not required: a search whose
    # worklist stays below its threshold donates every child and pushes none.)
    for slot in ("snapshot", "degree_one_scans", "triangle_scans", "removals", "stop_checks", "argmax",
                 "donate_or_push", "take_v", "take_neighbourhood", "acquire"):
        assert r["cycle_share"][slot] > 0, (which, slot)
    assert r["passes"]["degree_one_passes"] > 0 and r["passes"]["triangle_passes"] > 0
    # Pass counts of the three rules add up to the product's rule-pass counter.
    assert sum(r["passes"].values()) == r["rule_passes"]
    # Traced time and cycles of each worker's first thread fit inside the launch (workers x duration).
    span_ns = r["kernel_ms"] * 1e6
    assert 0 < r["worker_ns_total"] <= r["workers"] * span_ns * 1.02
    assert 0 < r["cycles_total"] <= r["workers"] * span_ns * 1e-9 * sm_max_hz() * 1.02
    assert abs(sum(r["time_share"].values()) - 1.0) < 1e-9
    assert abs(sum(r["cycle_share"].values()) - 1.0) < 1e-9
    assert r["time_share"]["reduction_rules_and_stop_check"] > 0 and r["time_share"]["branching"] > 0
    load = r["sm_load"]
    assert load is not None and load["sms"] > 0 and load["min_over_mean"] <= 1.0 <= load["max_over_mean"]
