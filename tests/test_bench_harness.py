"""The multi-rank harness of bench.py on CPU: two gloo ranks, barrier and the
max-over-ranks reduction used for the timed region (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d, r, ws, local = bench._dist()
    assert (r, ws, local) == (rank, world, rank)
    bench.barrier(d)
    m = bench.max_over_ranks(d, 10.0 + 5.0 * rank)
    out[rank] = m
    d.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 15.0


def test_single_process_has_no_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    d, r, ws, local = bench._dist()
    assert d is None and ws == 1
    assert bench.max_over_ranks(None, 3.5) == 3.5
