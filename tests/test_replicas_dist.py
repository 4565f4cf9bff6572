"""Multi-process host logic (replicas only) with the gloo backend on CPU, world size 2.

Each rank builds its own ensemble (different seeds, same replica sizes), the job time is the max
over ranks, and the job throughput counts every rank's particle-steps.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_1506_05094_gb300 import replicas as rep

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = rep.rank_ensemble(rank, replicas=3)
        ms = 10.0 + 5.0 * rank                       # pretend rank 1 is slower
        ms_max = rep.max_over_ranks(ms)
        n = wl.n_total
        out[rank] = (ms_max, [s.n for s in wl.states], float(wl.states[0].pos[0, 0]),
                     rep.job_throughput(n, world, 100, ms_max), n)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a multi-threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (ms0, sizes0, x0, v0, n0), (ms1, sizes1, x1, v1, n1) = res[0], res[1]
    assert ms0 == ms1 == 15.0                          # both see the slowest rank's time
    assert sizes0 == sizes1 and n0 == n1               # same per-GPU work (weak scaling)
    assert x0 != x1                                    # different initial configurations
    assert v0 == pytest.approx(n0 * 2 * 100 / 0.015)  # whole-job particle-steps / max time


def test_single_process_is_identity():
    from paper_1506_05094_gb300 import replicas as rep

    assert rep.max_over_ranks(3.5) == 3.5
    assert rep.rank_seed(1004, 0) == 1004 and rep.rank_seed(1004, 2) == 3004
