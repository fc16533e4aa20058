"""The multi-rank path of bench.py (independent replicas, weak scaling: no data-path
collective) on two gloo ranks on the CPU: the timed region is the slowest rank's, and the
whole-job rate counts every replica's work."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

_BENCH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", _BENCH)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    dist.barrier()
    got = b.max_over_ranks(ms, dist, "cpu")
    out[rank] = (got, b.replica_rate(world, 2e12, got * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # two replicas of 2e12 flops in 20 ms: 200,000 GFLOP/s for the whole job
    assert res[0][1] == pytest.approx(2 * 2e12 / 0.020 / 1e9)


def test_single_process_has_no_collective():
    b = _bench()
    assert b.max_over_ranks(3.5, None, "cpu") == 3.5
    assert b.replica_rate(1, 1e9, 1.0) == pytest.approx(1.0)
