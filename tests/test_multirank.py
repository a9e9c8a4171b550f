"""The N-replica path of the benchmark (queries sharded over ranks, no data-path collective): the
whole-job value is all ranks' queries over the slowest rank's time.  Runs as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [40.0, 50.0][rank]          # the second replica is slower
    value, ms = bench.aggregate(ms_local, 10_000, world)
    q.put((rank, value, ms))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms in got:
        assert ms == 50.0
        assert value == pytest.approx(2 * 10_000 / 0.050)


def test_single_replica_needs_no_process_group():
    value, ms = bench.aggregate(25.0, 1000, 1)
    assert ms == 25.0 and value == pytest.approx(40_000.0)
