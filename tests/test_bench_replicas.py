"""bench.py's replica aggregation with more than one rank, run as two gloo ranks on CPU: every rank
takes the slowest rank's time, and the whole-job value counts the nodes of all replicas."""
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms_max = bench.replica_max(10.0 * (rank + 1), world, "cpu")
        q.put((rank, ms_max, bench.replica_mlups(1000, 50, ms_max * 1e-3, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_are_timed_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r for r, _, _ in results] == [0, 1]
    for _, ms_max, value in results:
        assert ms_max == 20.0
        assert value == pytest.approx(2 * 1000 * 50 / 0.020 / 1e6)


def test_one_replica_is_its_own_time():
    assert bench.replica_max(7.5, 1, "cpu") == 7.5
    assert bench.replica_mlups(4194304, 5000, 1.0, 1) == pytest.approx(4194304 * 5000 / 1e6)
