"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

Events are independent, so N ranks each run their own events (weak scaling) with no
collective on the data path; the only collective is the max over ranks of the timed
duration. These tests run that logic with world size 2 on the gloo backend."""

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
    import torch.distributed as dist
    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = synth.generate_standard(50, bench.rank_workload_seed(rank))
        # each rank's own per-step time; the job time is the slowest rank's
        my_ms = 10.0 + rank
        slowest = bench.max_over_ranks(my_ms, world)
        out[rank] = (b.features[2, :5].tolist(), slowest,
                     bench.aggregate_value(50, world, 4, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_take_the_max():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    z0, slow0, v0 = res[0]
    z1, slow1, v1 = res[1]
    assert z0 != z1                       # distinct events per rank
    assert slow0 == slow1 == 11.0         # max over ranks
    assert v0 == v1 == pytest.approx(50 * 2 * 4 / 0.011)
