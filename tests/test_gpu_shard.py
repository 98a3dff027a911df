"""GPU parity of wst_image_range, the per-rank step of plane sharding: the partial image
of a plane range against the oracle's image of the visibilities in those planes, and
the sum of the partial images of a partition of the planes against wst_image."""
import numpy as np
import pytest

import oracle
from oracle import OracleConfig
from paper_2301_06061_gb300 import shard, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def wst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06061_gb300 import build, wst as w

    build.build()
    w.load_library()
    return w


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(gpu, ref):
    return float(np.abs(np.asarray(gpu, np.complex128) - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("n,n_w,chunk,world", [(256, 8, 0, 3), (256, 8, 3, 2), (1024, 5, 2, 4), (4096, 6, 0, 2)])
def test_plane_ranges_sum_to_the_whole_image(wst, n, n_w, chunk, world):
    rng = np.random.default_rng(n + world)
    u, v, w = synth.disk_uvw(6000, 0.45 * n / 0.1, 200.0, rng)
    vis = synth.random_visibilities(u.size, rng)
    cfg = wst.Config(n=n, fov=0.1, n_w=n_w, w_min=-200.0, w_max=200.0, planes_per_chunk=chunk)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    whole = plan.image()[0].cpu().numpy().astype(np.complex128)
    ocfg = OracleConfig(n, 0.1, n_w, -200.0, 200.0, 7)
    k, _, _, _ = oracle.locate(ocfg, u, v, w, vis)
    total = np.zeros((n, n), np.complex128)
    for b, e in shard.plane_ranges(n_w, world):
        part = plan.image_range(b, e)[0].cpu().numpy().astype(np.complex128)
        m = shard.owned(k, b, e)
        if m.any():
            ref = oracle.image(ocfg, u[m], v[m], w[m], vis[m], correct=False)
            unc = plan.image_range(b, e, flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
            assert rel_err(unc, ref) < TOL
        total += part
    assert rel_err(total, whole) < TOL


def test_ranges_across_images_of_a_batch(wst):
    """Batch of 3 images x 4 planes: a range that ends inside image 0, one that spans the
    end of image 0 and the start of image 1, and one over image 2 only; images outside a
    range are zero."""
    n, n_w = 256, 4
    rng = np.random.default_rng(31)
    counts = [1500, 2500, 900]
    us, vs, ws, vv = [], [], [], []
    for c in counts:
        a, b_, c_ = synth.disk_uvw(c, 0.45 * n / 0.1, 150.0, rng)
        us.append(a); vs.append(b_); ws.append(c_); vv.append(synth.random_visibilities(c, rng))
    off = np.concatenate([[0], np.cumsum(counts)])
    plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=n_w, w_min=-150.0, w_max=150.0, batch=3, planes_per_chunk=3))
    plan.set_vis(dev(np.concatenate(us)), dev(np.concatenate(vs)), dev(np.concatenate(ws)),
                 dev(np.concatenate(vv)), None, [int(x) for x in off])
    whole = plan.image().cpu().numpy().astype(np.complex128)
    ocfg = OracleConfig(n, 0.1, n_w, -150.0, 150.0, 7)
    total = np.zeros_like(whole)
    for b, e in ((0, 2), (2, 6), (6, 8), (8, 12)):
        part = plan.image_range(b, e).cpu().numpy()
        for i in range(3):
            lo, hi = max(b, i * n_w), min(e, (i + 1) * n_w)
            if lo >= hi:
                assert np.all(part[i] == 0)
                continue
            k, _, _, _ = oracle.locate(ocfg, us[i], vs[i], ws[i], vv[i])
            m = shard.owned(k, lo - i * n_w, hi - i * n_w)
            ref = oracle.image(ocfg, us[i][m], vs[i][m], ws[i][m], vv[i][m])
            assert rel_err(part[i][64:192, 64:192], ref[64:192, 64:192]) < TOL
        total += part
    assert rel_err(total, whole) < TOL
    empty = plan.image_range(5, 5)
    assert torch.count_nonzero(empty).item() == 0
