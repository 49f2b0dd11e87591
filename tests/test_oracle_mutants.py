"""The pins must be strong enough to catch plausible mistakes in the oracle.

Each mutant is a copy of oracle/vc_oracle.c with one planted mistake (a dropped term, a flipped
comparison, an off-by-one threshold, a dropped tie-break), compiled on the CPU into a temporary
library; the pin battery of test_oracle_pins must report at least one failure for it.  The battery
runs in a child process with a time limit: a mutant that hangs or crashes counts as caught too.
"""
import os
import subprocess
import sys

import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "vc_oracle.c")

MUTANTS = [
    ("degree-one tie-break takes the larger id",
     "if (x->deg[u] == 1 && u > v) continue;", "if (x->deg[u] == 1 && u < v) continue;"),
    ("degree-one tie-break dropped",
     "if (x->deg[u] == 1 && u > v) continue;", ";"),
    ("triangle tie-break dropped",
     "if ((x->deg[u] == 2 && u < v) || (x->deg[w] == 2 && w < v)) continue;", ";"),
    ("triangle adjacency test dropped",
     "if (!adjacent(g, u, w)) continue;", ";"),
    ("MVC high-degree threshold one too low",
     "? bound - x->S - 1 : bound - x->S;", "? bound - x->S - 2 : bound - x->S;"),
    ("PVC high-degree threshold one too low",
     "? bound - x->S - 1 : bound - x->S;", "? bound - x->S - 1 : bound - x->S - 1;"),
    ("edge bound prunes at equality",
     "return x->m > t * t;", "return x->m >= t * t;"),
    ("MVC size bound only prunes above best",
     "if (x->S >= bound) return 1;", "if (x->S > bound) return 1;"),
    ("edges between two removed vertices not subtracted",
     "x->m -= 1; /* edge between two removed vertices: count it once */", ";"),
    ("edges between two removed vertices subtracted twice",
     "} else if (u > v) {", "} else {"),
    ("neighbour degrees not decremented",
     "x->deg[u] -= 1; /* edge vu leaves the graph */", ";"),
    ("N(v) branch skipped",
     "if (x->deg[g->adj[e]] != REMOVED) s->mark[g->adj[e]] = 1;", ";"),
    ("PVC greedy shortcut accepts a cover one too large",
     "if (u <= k) { /* reading R6 */", "if (u <= k + 1) { /* reading R6 */"),
    ("maximum-degree ties go to the highest id",
     "        if (x->deg[v] > best_d) {", "        if (x->deg[v] >= best_d) {"),
    ("greedy skips the degree-two-triangle rule",
     "        reduce(&g, &x, mark, ORC_MVC, 0, RULE_DEG1 | RULE_DEG2TRI);",
     "        reduce(&g, &x, mark, ORC_MVC, 0, RULE_DEG1);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib), str(mutated)], check=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; import oracle; from tests.test_oracle_pins import run_pins; "
            f"f = run_pins(oracle.Oracle({str(lib)!r}), quick=True); print(len(f)); sys.exit(0)")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=20)
    except subprocess.TimeoutExpired:
        return  # caught: the mutant never finishes the battery
    if r.returncode != 0:
        return  # caught: the mutant crashed
    assert int(r.stdout.strip().splitlines()[-1]) > 0, f"pins did not catch mutant: {name}"
