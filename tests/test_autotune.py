"""Autotuner search logic (CPU, fake measurements) and one GPU tuning run on a small batch."""
import math
import os

import pytest

from paper_2204_10402_gb300 import autotune


def test_coordinate_descent_finds_separable_minimum():
    # A separable cost with a known minimum: the search must reach it and never re-measure.
    target = {"worker_threads": 64, "width": 16, "donate_threshold": 1.0, "worklist_capacity": 262144,
              "stage_csr": -1}
    calls = []

    def measure(cfg):
        calls.append(cfg)
        full = {"worker_threads": 32, "width": 16, "donate_threshold": 0.5, "worklist_capacity": 262144,
                "stage_csr": 0}
        full.update(cfg)
        return 100.0 + sum(abs(math.log2(full[k] + 2) - math.log2(v + 2)) * 10 for k, v in target.items())

    cfg, ms, trials = autotune.coordinate_descent(measure, {})
    full = {"worker_threads": 32, "width": 16, "donate_threshold": 0.5, "worklist_capacity": 262144, "stage_csr": 0}
    full.update(cfg)
    assert full == target
    assert ms == pytest.approx(100.0)
    assert len(calls) == len({str(sorted(c.items())) for c in calls})


def test_rejected_configs_are_skipped():
    def measure(cfg):
        return float("inf") if cfg.get("width") == 32 else 1.0 + (cfg.get("worker_threads", 32) == 32)
    cfg, ms, _ = autotune.coordinate_descent(measure, {})
    assert cfg.get("width", 16) == 16 and ms == 1.0


def test_size_classes_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("VC_AUTOTUNE_CACHE", str(tmp_path / "t.json"))
    assert autotune.size_class(60) == 64 and autotune.size_class(120) == 128 and autotune.size_class(3000) == 4096
    autotune.save_cache({"dev": {"batch:128": {"config": {"worker_threads": 32}, "ms": 1.0}}})
    assert autotune.load_cache()["dev"]["batch:128"]["ms"] == 1.0


@pytest.mark.gpu
def test_tune_small_batch(tmp_path, monkeypatch):
    import torch
    import paper_2204_10402_gb300 as vc
    from paper_2204_10402_gb300 import build
    from paper_2204_10402_gb300 import graphs as G
    build.build()
    vc.load()
    monkeypatch.setenv("VC_AUTOTUNE_CACHE", str(tmp_path / "t.json"))
    b = G.batch_gnp(256)
    off = torch.from_numpy(b.offsets).cuda()
    nbr = torch.from_numpy(b.neighbors).cuda()
    space = {"worker_threads": (32, 64), "donate_threshold": (0.5, 1.0), "stage_csr": (0, -1)}
    cfg, ms, trials = autotune.tune_batch(b.vtx, b.edge, off, nbr, repeats=1, sweeps=1, space=space)
    assert math.isfinite(ms) and len(trials) >= 3
    got = autotune.config_for(120)
    assert got is not None
    sizes, _, _ = vc.mvc_batch(b.vtx, b.edge, off, nbr, config=got, want_covers=False)
    ref, _, _ = vc.mvc_batch(b.vtx, b.edge, off, nbr, want_covers=False)
    assert list(sizes) == list(ref)
    # Both against the oracle's stored answers for the same 256 graphs (tests/golden, oracle only).
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096_mvc.txt")
    want = [int(l.split()[3]) for l in open(gold) if not l.startswith("#")][:256]
    assert list(sizes) == want
