"""vc_mvc_noalloc: the allocation-free MVC entry point, for callers whose device memory belongs to
a pool or arena or whose request path may not call cudaMalloc/cudaFree.

It is checked through the C ABI against vc_mvc (the allocating entry point) on the same device
inputs, twice in a row per graph: the answers are integers and must be equal, and both covers must
verify.  The second call exercises the reuse of the one scratch array that all calls share.  This
file is collected last so that a run stopping at its first failure has run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2204_10402_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vc():
    import torch
    assert torch.cuda.is_available()
    import paper_2204_10402_gb300 as vc
    from paper_2204_10402_gb300 import build
    build.build()
    vc.load()
    return vc


def graphs():
    out = [G.gnp(60, 0.10, 0), G.petersen(), G.path(9)]
    out += [G.gnp(n, p, 300 + i, draw_offset=2) for i, (n, p) in enumerate([(40, 0.3), (100, 0.12), (120, 0.2)])]
    out.append(G.gnp_with_planted_clique(160, 0.05, 10, 0)[0])
    out.append(G.chung_lu(500, 6.0, 3))
    return out


def test_noalloc_matches_allocating_entry_point(vc):
    import torch
    for g in graphs():
        off = torch.from_numpy(g.offsets).cuda()
        nbr = torch.from_numpy(g.neighbors).cuda()
        ref = vc.mvc(off, nbr)
        for _ in range(2):  # two calls in a row share and reuse the scratch array
            a = vc.mvc_noalloc(off, nbr)
            assert a.value == ref.value, (g.n, g.m, a.value, ref.value)
            cover = a.cover.cpu().numpy().astype(bool)
            assert cover.sum() == a.value
            assert oracle.verify_cover(g, cover)
            assert a.stats["stack_depth"] > 0 and a.stats["width"] == 16


def test_noalloc_rejects_settings_it_cannot_honour(vc):
    import torch
    g = G.gnp(60, 0.10, 0)
    off, nbr = torch.from_numpy(g.offsets).cuda(), torch.from_numpy(g.neighbors).cuda()
    want = vc.mvc(off, nbr).value
    for bad in (dict(width=32), dict(bit_rows=1), dict(stage_csr=1), dict(node_in_global=1),
                dict(worklist_capacity=4096)):
        with pytest.raises(vc.VCError) as e:
            vc.mvc_noalloc(off, nbr, config=vc.make_config(**bad))
        assert e.value.code == vc.VC_EINVAL, bad
    for ok in (dict(width=16), dict(stage_csr=-1), dict(worklist_capacity=1024), dict(donate_threshold=-1.0),
               dict(donate_threshold=1.0)):
        assert vc.mvc_noalloc(off, nbr, config=vc.make_config(**ok)).value == want, ok


def test_noalloc_rejects_oversize_and_host_inputs(vc):
    import torch
    big = G.gnp(vc.NOALLOC_MAX_N + 1, 0.01, 5)
    with pytest.raises(vc.VCError) as e:
        vc.mvc_noalloc(torch.from_numpy(big.offsets).cuda(), torch.from_numpy(big.neighbors).cuda())
    assert e.value.code == vc.VC_EINVAL
    g = G.petersen()
    with pytest.raises(ValueError):
        vc.mvc_noalloc(g.offsets, g.neighbors)


def test_noalloc_calls_from_several_threads_are_serialised(vc):
    # Four host threads, each on its own stream, call concurrently (ctypes releases the GIL); the
    # library serialises them on the one scratch array, so every answer equals the oracle's.
    import threading
    import torch
    gs = graphs()[:6]
    want = [oracle.mvc(g)[0] for g in gs]
    dev = [(torch.from_numpy(g.offsets).cuda(), torch.from_numpy(g.neighbors).cuda()) for g in gs]
    torch.cuda.synchronize()
    errors = []

    def work(t):
        try:
            s = torch.cuda.Stream()
            for _ in range(3):
                for i in range(len(gs)):
                    j = (i + t) % len(gs)
                    a = vc.mvc_noalloc(*dev[j], stream=s)
                    cover = a.cover.cpu().numpy().astype(bool)
                    if a.value != want[j] or cover.sum() != a.value or not oracle.verify_cover(gs[j], cover):
                        errors.append((t, j, a.value, want[j]))
        except Exception as e:  # reported below, in the test's own thread
            errors.append((t, repr(e)))

    threads = [threading.Thread(target=work, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=120)
    assert not any(th.is_alive() for th in threads)
    assert not errors, errors
