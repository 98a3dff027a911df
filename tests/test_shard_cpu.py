"""Plane sharding on CPU: the split of the w-planes over ranks and the one all-reduce of
the partial images, run as two (and three) gloo ranks with the FP64 oracle standing in
for each rank's GPU (the partial image of a plane range is the oracle image of the
visibilities the oracle places in those planes, with the same plane geometry).  The
reduced image equals the single-rank image.  The GPU side (``wst_image_range``) is
checked in tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2301_06061_gb300 import shard, synth  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    work = synth.tiny(n_vis=3000, n=64, n_w=7)
    vis = synth.random_visibilities(work.n_vis, np.random.default_rng(5))
    return work, vis


def _partial_image(rank: int, world: int):
    """This rank's partial image: the oracle stands in for the GPU's wst_image_range."""
    import oracle
    from oracle import OracleConfig

    work, vis = _case()
    cfg = OracleConfig(work.n, work.fov, work.n_w, work.w_min, work.w_max, work.support, "gauss", 0.875)
    k, _, _, _ = oracle.locate(cfg, work.u, work.v, work.w, vis)
    b, e = shard.plane_ranges(work.n_w, world)[rank]
    m = shard.owned(k, b, e)
    return oracle.image(cfg, work.u[m], work.v[m], work.w[m], vis[m]), int(m.sum())


def _rank_main(rank: int, world: int, port: int, queue) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img, n_own = _partial_image(rank, world)
        t = torch.from_numpy(img.astype(np.complex128))
        shard.reduce_images(t, dist)
        queue.put((rank, t.numpy(), n_own))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reduce_plane_ranges_to_the_single_rank_image(world):
    import oracle
    from oracle import OracleConfig

    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, queue)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        results = sorted((queue.get(timeout=180) for _ in procs), key=lambda x: x[0])
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    work, vis = _case()
    cfg = OracleConfig(work.n, work.fov, work.n_w, work.w_min, work.w_max, work.support, "gauss", 0.875)
    whole = oracle.image(cfg, work.u, work.v, work.w, vis)
    _, _, _, st = oracle.locate(cfg, work.u, work.v, work.w, vis)
    # every kept visibility is owned by exactly one rank
    assert sum(r[2] for r in results) == int((st == 0).sum())
    for _, img, _ in results:  # every rank holds the reduced image
        assert np.abs(img - whole).max() <= 1e-12 * np.abs(whole).max()


def test_plane_ranges_partition_the_planes():
    for n_planes in (0, 1, 7, 32, 1024):
        for world in (1, 2, 3, 8):
            r = shard.plane_ranges(n_planes, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == n_planes
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [e - b for b, e in r]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard.plane_ranges(4, 0)


def test_owned_excludes_dropped_visibilities():
    k = np.array([-1, 0, 3, 4, 6, -1])
    assert shard.owned(k, 3, 5).tolist() == [False, False, True, True, False, False]
    assert shard.owned(k, 0, 7).sum() == 4


def test_single_process_reduce_is_a_no_op():
    t = torch.ones(3, dtype=torch.complex64)
    shard.reduce_images(t, None)
    assert torch.equal(t, torch.ones(3, dtype=torch.complex64))
