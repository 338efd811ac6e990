"""The multi-replica bookkeeping of bench.py on CPU: two gloo ranks, each
with its own replica of the workload; the whole-job value is all ranks'
units over the slowest rank's time (weak scaling, no collective on the data
path)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    assert bench.dist_env() == (rank, world, rank)
    bench.dist_init(world, "gloo")
    # rank r processed 1000 units in (r + 1) seconds
    value, t = bench.aggregate(1000.0, float(rank + 1), world)
    mx = bench.reduce_max(float(10 * rank), world)
    bench.barrier(world)
    out[rank] = (value, t, mx)
    dist.destroy_process_group()


def test_two_gloo_replicas_report_units_over_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t, mx = res[rank]
        assert t == 2.0                      # the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 2.0)
        assert mx == 10.0


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(100.0, 4.0, 1) == (25.0, 4.0)
