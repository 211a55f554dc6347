"""Replica scaling logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

Every rank runs its own copy of the workload (weak scaling); the whole-job
value is the blocks of all ranks over the slowest rank's time.  No
collective touches the data path -- only the timing reduction does."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    d = bench.Dist("gloo")
    d.barrier()
    # rank r processed (r + 1) * 1000 blocks per step in (r + 1) * 10 ms
    value, ms, blocks = bench.aggregate(d, (rank + 1) * 1000, (rank + 1) * 10.0, steps=4)
    out[rank] = (value, ms, blocks)
    d.barrier()
    d.close()


def test_two_rank_replicas_aggregate_over_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    # total blocks 3000 per step, 4 steps, slowest rank 20 ms
    for r in range(world):
        value, ms, blocks = out[r]
        assert ms == pytest.approx(20.0)
        assert blocks == pytest.approx(3000.0)
        assert value == pytest.approx(3000 * 4 / 0.020)


def test_single_process_aggregate_is_identity():
    import bench

    class One:
        def max(self, v):
            return v

        def sum(self, v):
            return v

    value, ms, blocks = bench.aggregate(One(), 500, 5.0, steps=2)
    assert (value, ms, blocks) == (500 * 2 / 0.005, 5.0, 500)
