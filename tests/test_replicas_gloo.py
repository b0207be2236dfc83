"""The multi-GPU form is N independent replicas (the path exchanges nothing between runs):
bench.py's whole-job aggregation takes the slowest rank's time and the sum of the units
all ranks processed. Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [10.0 + 5.0 * rank, 3.0 - rank]
    counts = [1000 * (rank + 1), 7]
    t, c = bench.aggregate_replicas(dist, times, counts, "cpu")
    out[rank] = (t, c)
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        t, c = out[r]
        assert t == [15.0, 3.0]  # max over ranks
        assert c == [3000.0, 14.0]  # sum over ranks


def test_replica_aggregation_single_process():
    import bench

    t, c = bench.aggregate_replicas(None, [1.5, 2.0], [10, 20], "cpu")
    assert t == [1.5, 2.0] and c == [10.0, 20.0]
