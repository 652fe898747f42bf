"""The N > 1 path of bench.py (replicas only: a barrier, the slowest rank's time,
whole-job bytes), run as two gloo ranks on the CPU; and the reference arm, which
only rank 0 runs."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slowest
    total = bench.max_over_ranks(local_ms, "cpu", world)
    q.put((rank, total, bench.job_value(1_000_000_000, 2, total, world)))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, total, value in got:
        assert total == 20.0
        assert abs(value - 2 * 1e9 * 2 / 0.02 / 1e9) < 1e-9  # 2 replicas x 2 steps x 1 GB in 20 ms


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, "cpu", 1) == 12.5
    assert bench.job_value(4e9, 10, 20.0, 1) == 4e9 * 10 / 0.02 / 1e9


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    assert buf.getvalue() == ""
