"""The multi-GPU form of the benchmark runs independent replicas (one solve per rank,
no collective on the data path) and reports units over all ranks divided by the
slowest rank's time.  Checked here with two gloo processes on the CPU."""
import os
import socket

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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1200.0, 1500.0][rank]          # rank 1 is the slower replica
    value, ms = bench.replica_throughput(local_ms, units_per_rank=7_680_000 * 100)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, ms = res[rank]
        assert ms == 1500.0                     # max over ranks
        assert value == pytest.approx(2 * 7_680_000 * 100 / 1.5)


def test_single_process_is_identity():
    import bench
    value, ms = bench.replica_throughput(250.0, 1000)
    assert ms == 250.0 and value == pytest.approx(4000.0)
