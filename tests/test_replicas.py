"""Multi-GPU runs are replicas (each rank evolves its own hierarchy, no
collective on the data path): the bench's host-side aggregation -- the
slowest rank's time by one all-reduce, the whole-job zone-updates/s -- on two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 25.0 * rank  # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, dist)
    out[rank] = (ms, bench.whole_job_value(77758464, world, ms))
    dist.destroy_process_group()


def test_two_replicas_max_time_and_whole_job_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 125.0
    assert res[0][1] == pytest.approx(2 * 77758464 / 0.125)


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.whole_job_value(1000, 1, 1.0) == pytest.approx(1e6)
