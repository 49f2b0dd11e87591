"""Register and spill budgets of the traversal kernels, from ptxas's resource report (CPU only).

The library build compiles every translation unit with ``-Xptxas -v`` and keeps the report in
``_build/ptxas.log``.  The traversal is issue-bound, so a change that makes a hot instance spill
or outgrow its register budget costs throughput at once: for example a flag kept live across the
traversal loop once added 60-100 bytes of spills to the CSR-walk workers (planted clique n = 160:
6.2 -> 6.9 ms).  The limits below are the instances' current figures with a little headroom.
"""
import os
import re

import pytest

from paper_2204_10402_gb300 import build

LOG = os.path.join(build.BUILD, "ptxas.log")


def resources() -> dict:
    if not os.path.exists(LOG):
        build.build(force=True)
    else:
        build.build()
    out, cur = {}, None
    for line in open(LOG):
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            cur = m.group(1)
            out[cur] = {"regs": None, "spill_st": 0, "spill_ld": 0}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            out[cur]["spill_st"], out[cur]["spill_ld"] = int(m.group(1)), int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            out[cur]["regs"] = int(m.group(1))
    return out


def traverse(width_char: str, wt: int, nw: int, serve: bool) -> str:
    # vc::traverse_kernel<W, WT, GM=false, NW, SERVE>(vc::Params), W = int ('i') or short ('s')
    return f"_ZN2vc15traverse_kernelI{width_char}Li{wt}ELb0ELi{nw}ELb{int(serve)}EEEvNS_6ParamsE"


@pytest.fixture(scope="module")
def res():
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return resources()


@pytest.mark.parametrize("w", ["i", "s"])
def test_batch_bit_row_instance_fits_its_budget(res, w):
    # the 4096-graph batch's kernel: 64-register cap (32 one-warp workers per SM), no spills
    r = res[traverse(w, 32, 4, False)]
    assert r["regs"] <= 64 and r["spill_st"] == 0 and r["spill_ld"] == 0, r


@pytest.mark.parametrize("w", ["i", "s"])
def test_eight_word_instance_fits_its_budget(res, w):
    # launch bounds (32, 28): at most 72 registers; its spills stay small
    r = res[traverse(w, 32, 8, False)]
    assert r["regs"] <= 72 and r["spill_st"] <= 128, r


def test_serving_bit_row_instance_fits_its_budget(res):
    r = res[traverse("i", 32, 4, True)]
    assert r["regs"] <= 64 and r["spill_st"] == 0, r


@pytest.mark.parametrize("wt,limit", [(32, 64), (64, 72), (128, 24), (256, 24), (512, 24)])
def test_csr_walk_instances_spill_little(res, wt, limit):
    r = res[traverse("i", wt, 0, False)]
    assert r["regs"] <= 64 and r["spill_st"] <= limit, (wt, r)


@pytest.mark.parametrize("wt", [64, 128, 256, 512])
def test_serving_csr_walk_instances_do_not_spill(res, wt):
    # the server's CSR-walk workers (256 threads by default)
    r = res[traverse("i", wt, 0, True)]
    assert r["regs"] <= 64 and r["spill_st"] <= 8, (wt, r)
