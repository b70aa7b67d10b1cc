"""The multi-rank aggregation of bench.py (replicas, one per GPU) on CPU ranks
with the gloo backend: the whole-job value is the units of all ranks over the
slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 250.0][rank]
    units = [1.0e9, 3.0e9][rank]
    q.put((rank, bench.reduce_over_ranks(ms, units, "cpu", world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_max_time_and_sum_units():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        ms, units, value = out[r]
        assert ms == 250.0 and units == 4.0e9
        assert value == pytest.approx(4.0e9 / 0.25)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(200.0, 2.0e9, "cpu", 1) == (200.0, 2.0e9, 1.0e10)
