"""The multi-rank path of bench.py on CPU: replicas, one rank per GPU, weak scaling.

No exchange step exists on the data path (every rank images its own visibilities), so
the only cross-rank operations are the barriers around the timed region and the
maximum of the per-step times.  Two gloo ranks exercise them here; the reference arm
runs on rank 0 only.
"""
import os
import socket
from types import SimpleNamespace

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, queue) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")  # rank 1 is the slower one
        dist.barrier()
        queue.put((rank, ms, bench.job_mvis(world, 1_000_000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_sum_the_work():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(queue.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[0] for r in results] == [0, 1]
    assert [r[1] for r in results] == [15.0, 15.0]  # both ranks report the slowest time
    # 2 ranks x 1e6 visibilities in 15 ms
    assert results[0][2] == pytest.approx(2 * 1_000_000 / 15e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_mvis(1, 1_000_000, 10.0) == pytest.approx(100.0)


def test_ranks_image_different_seeded_workloads():
    """Weak scaling: each rank's workload has the same shape and its own seed."""
    w0, w1 = bench.make_workload("array", 0), bench.make_workload("array", 1)
    assert w0.n_vis == w1.n_vis and w0.n == w1.n and w0.n_w == w1.n_w
    assert not np.array_equal(w0.u, w1.u)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = SimpleNamespace(workload="large", steps=1, warmup=0)
    bench.run_reference(args, rank=1, world=2)  # returns before any work
    assert capsys.readouterr().out == ""
