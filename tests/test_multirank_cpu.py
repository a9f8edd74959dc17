"""The multi-process logic of bench.py on CPU with the gloo backend (world size 2):
each rank gets its own independent field of the same size (weak scaling, no data
exchanged), and the job time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    wl = W.config("tiny")
    f = bench.rank_field(wl, rank)
    t = bench.max_over_ranks(1.0 + rank)  # rank r took 1 + r seconds
    out[rank] = (t, float(f.xy.sum()), f.n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_and_max_time():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.0          # max over ranks
    assert out[0][2] == out[1][2]                 # same size per rank
    assert out[0][1] != out[1][1]                 # independent fields
