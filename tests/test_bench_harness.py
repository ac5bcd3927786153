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


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the contract's keys; no GPU is involved."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "c0",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         env={k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK")})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
