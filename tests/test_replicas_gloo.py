"""The multi-GPU path of the benchmark is N independent replicas (the solve
does not shard): the timed region is the maximum over ranks and the value
counts every rank's bytes.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_setup()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, value = bench.aggregate(10.0 + 5.0 * rank, 10**9, 2, w)
        out[rank] = (w, r, local, t, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, local, t, value = res[rank]
        assert (w, r, local) == (world, rank, rank)
        assert t == 15.0
        assert value == pytest.approx(10**9 * 2 * world / 0.015 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    t, value = bench.aggregate(4.0, 2 * 10**9, 3, 1)
    assert t == 4.0 and value == pytest.approx(2 * 3 / 0.004)
