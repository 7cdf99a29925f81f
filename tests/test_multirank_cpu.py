"""The multi-process path of bench.py on CPU: two gloo ranks, each with its
own seeded replica input (no data-path collective), and the job time taken
as the maximum over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = dict(bench.WORKLOADS["line_2p20_c64"], d=10)
    x, _ = bench.make_input(wl, rank)
    t = bench.max_over_ranks([10.0 * (rank + 1), 1.0 + rank], "cpu")
    lines = bench.make_batch(dict(bench.WORKLOADS["batch_256_c64"], nlines=4, dmin=6, dmax=7), rank)
    out[rank] = (x[:8].copy(), t, [ln["x"][:4].copy() for ln in lines])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    import torch.multiprocessing as mp
    port = _free_port()
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        assert res[r][1] == [20.0, 2.0]           # max over ranks, seen by every rank
    # replicas: each rank draws its own input from the seeded generator
    assert not np.array_equal(res[0][0], res[1][0])
    assert not np.array_equal(res[0][2][0], res[1][2][0])
