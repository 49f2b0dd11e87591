"""The multi-GPU path of bench.py is replicas of independent batches: each rank solves its own
graphs and the ranks exchange only the timing maximum and the solve count.  Checked here with two
gloo ranks on CPU (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import torch.distributed as dist

    import bench
    from paper_2204_10402_gb300 import graphs as G
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    b = bench.workload(rank, 8)
    seeds = [rank * bench.NUM_GRAPHS + g for g in range(8)]
    same = all(np.array_equal(gr.offsets, G.gnp(*G.batch_gnp_params(s), s, draw_offset=2).offsets)
               for gr, s in zip(b.graphs, seeds))
    t_max, solves = bench.combine(1.0 + rank, 8)
    out.put((rank, seeds, same, t_max, solves))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_combine():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, same0, t0, n0), (r1, s1, same1, t1, n1) = res
    assert same0 and same1
    assert not set(s0) & set(s1)           # disjoint graphs per rank
    assert t0 == t1 == 2.0                 # the slowest rank's time
    assert n0 == n1 == 16                  # solves of both ranks
