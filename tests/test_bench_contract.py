"""The benchmark's JSON line (host side, no GPU): the reference arm's keys and that both arms
name the same workload, metric and unit."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import bench
    assert line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["config"]["workload"] == bench.workload_name(bench.NUM_GRAPHS)


def test_traffic_figure_follows_the_profiled_sources():
    # bench.py reports DRAM traffic only while the traversal kernel's sources hash to the value the
    # committed ncu summary records (null after a kernel change until the next capture).
    sys.path.insert(0, ROOT)
    import bench
    v = bench.measured_per_node("dram_bytes_per_tree_node")
    assert v is None or v > 0
    assert bench.measured_per_node("no_such_figure") is None


def test_source_hash_follows_code_not_comments(tmp_path):
    # The profile stays matched when only comments or layout change, and not when code changes.
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2204_10402_gb300", "csrc")
    copy = tmp_path / "csrc"
    shutil.copytree(src, copy)
    base = bench.traversal_source_hash(str(copy))
    assert base == bench.traversal_source_hash()
    dev = copy / "vc_device.cuh"
    text = dev.read_text()
    dev.write_text("// a new comment\n/* and a block\n   comment */\n\n" + text.replace("\n", "\n\n", 5))
    assert bench.traversal_source_hash(str(copy)) == base
    anchor = "constexpr unsigned kFull = 0xffffffffu;"
    assert anchor in text
    dev.write_text(text.replace(anchor, "constexpr unsigned kFull = 0x7fffffffu;"))
    assert bench.traversal_source_hash(str(copy)) != base


def test_e2e_copy_bytes_follow_the_c_structs(tmp_path):
    # The e2e line's byte counts use the sizes of the records the library really copies: pinned
    # here to the C structs by compiling their sizes out of the library's own header.
    sys.path.insert(0, ROOT)
    import bench
    from paper_2204_10402_gb300 import graphs as G
    src = tmp_path / "sizes.cpp"
    src.write_text('#include <cstdio>\n#include "vc_internal.h"\n'
                   'int main() { std::printf("%zu %zu %d\\n", sizeof(vc::Problem), sizeof(vc::Control), '
                   '(int)vc::kSmSlots); }\n')
    exe = tmp_path / "sizes"
    csrc = os.path.join(ROOT, "paper_2204_10402_gb300", "csrc")
    r = subprocess.run(["g++", "-std=c++17", "-I", csrc, "-o", str(exe), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    prob, ctrl, slots = map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split())
    assert (bench.PROBLEM_RECORD_BYTES, bench.CONTROL_BYTES, bench.SM_COUNTER_BYTES) == (prob, ctrl, 8 * slots)
    b = G.pack([G.path(3), G.petersen()])          # offsets 4 + 11 entries, neighbours 4 + 30
    h2d, d2h = bench.e2e_copy_bytes(b, 13)
    assert h2d == 4 * (15 + 34) + 2 * (prob + 8)
    assert d2h == 2 * prob + ctrl + 8 * slots + 4 * 13
    assert isinstance(h2d, int) and isinstance(d2h, int)
