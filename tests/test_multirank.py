"""The N>1 path of bench.py on CPU: two gloo ranks, each a replica, timed
with a barrier and aggregated as max time / total work (no data-path
collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.barrier()
    ms = [120.0, 200.0][rank]
    units = [3.0e12, 1.0e12][rank]
    t_max, value = bench.aggregate_over_ranks(ms, units, world)
    q.put((rank, t_max, value))
    dist.destroy_process_group()


def test_two_rank_replica_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in out:
        assert t_max == 200.0
        assert abs(value - 4.0e12 / 0.2) < 1e-3 * value


def test_single_rank_aggregation():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    t, v = bench.aggregate_over_ranks(50.0, 1e12, 1)
    assert t == 50.0 and abs(v - 2e13) < 1
