"""Multi-process host logic of bench.py (replicas, no data-path collective):
two gloo ranks on CPU agree on the max over ranks of the timed region and on
the whole-job value."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    m = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (m, bench.replica_value(world, 1000, 10, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_over_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 150.0
    assert v == pytest.approx(2 * 3 * 1000 * 10 / 0.150)
