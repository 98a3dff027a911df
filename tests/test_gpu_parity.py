"""GPU parity: every step of the CUDA path against the FP64 oracle, through the C ABI.

Tolerance: 1e-5 of the peak for FP32 results (planes, the image before the grid
correction U, and the corrected image D on the central half |nu| <= 1/4); over the
full corrected image the FP32 budget |dD| <= 1e-5 max|U| C_a C_b + 1e-6 |D|, because
the correction C_a C_b = 1/(Ghat(nu_a) Ghat(nu_b)) reaches ~2e3 (Gaussian, W=7) to
~8e3 (ES, W=8) at the corners of an unpadded grid and multiplies the FFT's uniform
rounding there.  Placement (plane, tap start) and counts are bit-exact.
"""
import numpy as np
import pytest

import oracle
from oracle import OracleConfig
from paper_2301_06061_gb300 import synth

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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_err(gpu, ref):
    ref = np.asarray(ref)
    scale = np.abs(ref).max()
    return float(np.abs(np.asarray(gpu, dtype=np.complex128) - ref).max() / max(scale, 1e-300))


def correction(ocfg):
    n = ocfg.n
    return 1.0 / oracle.kernel_ft(ocfg, (np.arange(n) - n // 2) / n)


def assert_image_parity(gpu, ref, ocfg, tol=TOL):
    """Corrected image: central half at tol of the peak; full image within the FP32 budget."""
    gpu = np.asarray(gpu, dtype=np.complex128)
    n = ref.shape[-1]
    cc = np.outer(correction(ocfg), correction(ocfg))
    u_peak = np.abs(ref / cc).max()
    err = np.abs(gpu - ref)
    c = slice(n // 4, 3 * n // 4)
    assert err[c, c].max() <= tol * np.abs(ref[c, c]).max(), err[c, c].max() / np.abs(ref[c, c]).max()
    budget = tol * u_peak * cc + 1e-6 * np.abs(ref)
    assert np.all(err <= budget), float((err / budget).max())


def make_case(n=256, fov=0.1, n_w=8, n_vis=3000, W=7, seed=0, radius=0.45, w_half=200.0):
    rng = np.random.default_rng(seed)
    u, v, w = synth.disk_uvw(n_vis, radius * n / fov, w_half, rng)
    vis = synth.random_visibilities(n_vis, rng)
    return u, v, w, vis


def ocfg_for(cfg, w_min, w_max, table=None):
    kern = {0: "gauss", 1: "es", 2: "table"}[cfg.kernel]
    return OracleConfig(cfg.n, cfg.fov, cfg.n_w, w_min, w_max, cfg.support, kern, cfg.kparam,
                        None if table is None else np.asarray(table, np.float64))


def gpu_plan(wst, cfg, u, v, w, vis, weight=None, offsets=None, table=None):
    plan = wst.Plan(cfg)
    if table is not None:
        plan.set_kernel_table(dev(np.asarray(table, np.float32)))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), None if weight is None else dev(weight), offsets)
    return plan


# ------------------------------------------------------------------------------------------
# K-S: placement is bit-exact
# ------------------------------------------------------------------------------------------

def test_vis_cells_bit_exact(wst):
    u, v, w, vis = make_case(n=256, n_vis=20000, radius=0.55, w_half=230.0)  # some dropped
    u[:5] = np.nan
    vis[5:8] = np.nan
    cfg = wst.Config(n=256, fov=0.1, n_w=8, w_min=-200.0, w_max=200.0)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    k = torch.empty(u.size, dtype=torch.int32, device="cuda")
    i0 = torch.empty_like(k)
    j0 = torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    ko, io, jo, st = oracle.locate(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis)
    np.testing.assert_array_equal(k.cpu().numpy(), ko)
    np.testing.assert_array_equal(i0.cpu().numpy(), io)
    np.testing.assert_array_equal(j0.cpu().numpy(), jo)
    s = plan.stats()
    assert s["n_kept"] == int((st == 0).sum())
    assert s["n_dropped"] == int((st == 1).sum()) > 0
    assert s["n_nonfinite"] == int((st == 2).sum()) == 8


def near_integer_coords(n, fov, W, rng, count=600):
    """u with half_n + u fov - W/2 on, or a few FP32 steps from, an integer tap start,
    including the tap starts where the drop rule switches (0 and n - W)."""
    m = np.concatenate([rng.integers(-3, n + 3, count - 8), [0, -1, 1, n - W, n - W + 1, n - W - 1, n // 2, 3]])
    u = ((m - n / 2 + W / 2) / fov).astype(np.float32)
    steps = rng.integers(-2, 3, m.size).astype(np.int32)
    out = u.copy()
    for k in range(1, 3):  # move by `steps` FP32 ulps
        out = np.where(steps >= k, np.nextafter(out, np.float32(np.inf)), out)
        out = np.where(steps <= -k, np.nextafter(out, np.float32(-np.inf)), out)
    return out


@pytest.mark.parametrize("n,fov,W", [(256, 0.1, 7), (16384, 0.5, 7), (4096, 0.2, 8)])
def test_vis_cells_near_decision_boundaries(wst, n, fov, W):
    """Tap starts and planes decided on or next to their boundaries agree bit for bit with
    the FP64 oracle (the float-float fast path must defer to FP64 there)."""
    rng = np.random.default_rng(n + W)
    u = near_integer_coords(n, fov, W, rng)
    v = rng.permutation(near_integer_coords(n, fov, W, rng))
    n_w, lo, hi = 8, -200.0, 200.0
    edges = lo + np.arange(n_w + 1) * (hi - lo) / n_w
    w = np.repeat(edges, -(-u.size // edges.size))[: u.size].astype(np.float32)
    steps = rng.integers(-2, 3, u.size)
    w = np.where(steps > 0, np.nextafter(w, np.float32(np.inf)), np.where(steps < 0, np.nextafter(w, np.float32(-np.inf)), w))
    w = rng.permutation(w.astype(np.float32))
    vis = np.ones(u.size, np.complex64)
    cfg = wst.Config(n=n, fov=fov, n_w=n_w, w_min=lo, w_max=hi, support=W, kparam=wst.DEFAULT_SIGMA[W],
                     planes_per_chunk=1)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    k = torch.empty(u.size, dtype=torch.int32, device="cuda")
    i0, j0 = torch.empty_like(k), torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    ko, io, jo, st = oracle.locate(ocfg_for(cfg, lo, hi), u, v, w, vis)
    np.testing.assert_array_equal(i0.cpu().numpy(), io)
    np.testing.assert_array_equal(j0.cpu().numpy(), jo)
    np.testing.assert_array_equal(k.cpu().numpy(), ko)
    s = plan.stats()
    assert s["n_kept"] == int((st == 0).sum()) and s["n_dropped"] == int((st == 1).sum()) > 0


def test_w_range_from_data(wst):
    u, v, w, vis = make_case(n=128, n_vis=5000)
    cfg = wst.Config(n=128, fov=0.1, n_w=5)  # w_min == w_max: from the data
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    lo, hi = oracle.resolve_w_range(w, 0.0, 0.0)
    s = plan.stats()
    assert s["w_min"] == lo and s["w_max"] == hi
    k = torch.empty(u.size, dtype=torch.int32, device="cuda")
    i0, j0 = torch.empty_like(k), torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    ko, _, _, _ = oracle.locate(ocfg_for(cfg, lo, hi), u, v, w, vis)
    np.testing.assert_array_equal(k.cpu().numpy(), ko)


def test_w_range_from_data_degenerate_single_w(wst):
    """Every w equal and the range from the data: the range is empty, every visibility
    goes to plane 0 (centre = that w), the other planes stay empty, and the image is the
    oracle's (one plane with its screen)."""
    u, v, _, vis = make_case(n=256, n_vis=3000, seed=77)
    w = np.full(u.size, 37.5, np.float32)
    cfg = wst.Config(n=256, fov=0.1, n_w=4)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    lo, hi = oracle.resolve_w_range(w, 0.0, 0.0)
    s = plan.stats()
    assert s["w_min"] == s["w_max"] == lo == hi == 37.5
    k = torch.empty(u.size, dtype=torch.int32, device="cuda")
    i0, j0 = torch.empty_like(k), torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    oc = ocfg_for(cfg, lo, hi)
    ko, _, _, _ = oracle.locate(oc, u, v, w, vis)
    np.testing.assert_array_equal(k.cpu().numpy(), ko)
    assert np.all(ko <= 0)  # plane 0 (a dropped visibility would read -1)
    img = plan.image()
    assert_image_parity(img[0].cpu().numpy(), oracle.image(oc, u, v, w, vis), oc)


# ------------------------------------------------------------------------------------------
# K-G: gridded planes
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,W", [(64, 7), (256, 7), (256, 8), (512, 5), (4096, 7)])
def test_grid_planes(wst, n, W):
    u, v, w, vis = make_case(n=n, n_vis=4000, seed=n + W)
    wt = np.random.default_rng(1).uniform(0.5, 2.0, u.size).astype(np.float32)
    cfg = wst.Config(n=n, fov=0.1, n_w=6, w_min=-200.0, w_max=200.0, support=W,
                     kparam=wst.DEFAULT_SIGMA.get(W, 0.8))
    plan = gpu_plan(wst, cfg, u, v, w, vis, weight=wt)
    g = torch.empty((6, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 6, g)
    ref = oracle.grid(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis, wt)
    assert rel_err(g.cpu().numpy(), ref) < TOL


def test_grid_dense_tile_collisions(wst):
    """Thousands of visibilities in one tile: shared-memory accumulation under contention."""
    rng = np.random.default_rng(3)
    n, fov = 256, 0.1
    u = rng.normal(0.0, 30.0, 20000).astype(np.float32)
    v = rng.normal(0.0, 30.0, 20000).astype(np.float32)
    w = rng.uniform(-10, 10, 20000).astype(np.float32)
    vis = synth.random_visibilities(20000, rng)
    cfg = wst.Config(n=n, fov=fov, n_w=2, w_min=-10.0, w_max=10.0)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    g = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 2, g)
    ref = oracle.grid(ocfg_for(cfg, -10.0, 10.0), u, v, w, vis)
    assert rel_err(g.cpu().numpy(), ref) < TOL


def test_grid_coherent_pileup_regrids_in_float(wst):
    """2000 identical visibilities on one cell centre, in a row whose other 8000
    visibilities spread over the columns: the row takes the fixed-point path (its busiest
    bin is not dominant), the pile-up exceeds the int32 range of the fine quantum, the
    kernel detects it and accumulates the row again in float; planes and image match the
    oracle."""
    rng = np.random.default_rng(13)
    n, fov, npile, nrow, nrest = 8192, 0.1, 2000, 8000, 3000  # fixed-point rows need n >= 8192
    u = np.concatenate([np.full(npile, 300.0), rng.uniform(-40000.0, 40000.0, nrow),
                        rng.uniform(-40000.0, 40000.0, nrest)]).astype(np.float32)
    v = np.concatenate([np.full(npile + nrow, -150.0), rng.uniform(-40000.0, 40000.0, nrest)]).astype(np.float32)
    w = rng.uniform(-10.0, 10.0, u.size).astype(np.float32)
    vis = np.concatenate([np.full(npile, 1.0 + 0.5j, np.complex64),
                          synth.random_visibilities(nrow + nrest, rng)]).astype(np.complex64)
    cfg = wst.Config(n=n, fov=fov, n_w=1, w_min=-10.0, w_max=10.0)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    g = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 1, g)
    oc = ocfg_for(cfg, -10.0, 10.0)
    assert rel_err(g.cpu().numpy(), oracle.grid(oc, u, v, w, vis)) < TOL
    img = plan.image(flags=wst.WST_NO_CORRECTION)
    assert rel_err(img[0].cpu().numpy(), oracle.image(oc, u, v, w, vis, correct=False)) < TOL


def test_grid_and_image_dense_rows_keep_float_atomics(wst):
    """A row whose busiest 64-column bin holds more than 8192 times the row's mean
    magnitude per visibility-row keeps float atomics (here 1.1M visibility-rows over seven
    bins); a plane holding such rows and ordinary (fixed-point) ones matches the oracle,
    gridded and imaged."""
    rng = np.random.default_rng(5)
    n, fov, nd, ns = 8192, 0.1, 1_100_000, 40000  # fixed-point rows need n >= 8192
    u = np.concatenate([rng.uniform(-2000.0, 2000.0, nd), rng.uniform(-40000.0, 40000.0, ns)]).astype(np.float32)
    v = np.concatenate([np.zeros(nd), rng.uniform(-40000.0, 40000.0, ns)]).astype(np.float32)
    w = rng.uniform(-10.0, 10.0, nd + ns).astype(np.float32)
    vis = synth.random_visibilities(nd + ns, rng)
    cfg = wst.Config(n=n, fov=fov, n_w=1, w_min=-10.0, w_max=10.0)  # rows 4093..4099: 1.1M each
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    g = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 1, g)
    oc = ocfg_for(cfg, -10.0, 10.0)
    assert rel_err(g.cpu().numpy(), oracle.grid(oc, u, v, w, vis)) < TOL
    img = plan.image(flags=wst.WST_NO_CORRECTION)
    assert rel_err(img[0].cpu().numpy(), oracle.image(oc, u, v, w, vis, correct=False)) < TOL


# ------------------------------------------------------------------------------------------
# K-F + K-P: transform, screen and plane sum; full image
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024, 2048])
def test_fft_correct_staged(wst, n):
    u, v, w, vis = make_case(n=n, n_vis=3000, seed=n)
    cfg = wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    g = torch.empty((4, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 4, g)
    img = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_fft_correct(plan.handle, 0, 2, g[0:2].contiguous(), img)
    wst.wst_fft_correct(plan.handle, 2, 4, g[2:4].contiguous(), img)
    ref = oracle.image(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis, correct=False)
    assert rel_err(img[0].cpu().numpy(), ref) < TOL
    wst.wst_correct(plan.handle, img)
    ref_c = oracle.image(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis, correct=True)
    assert_image_parity(img[0].cpu().numpy(), ref_c, ocfg_for(cfg, -200.0, 200.0))


@pytest.mark.parametrize("n,n_w,chunk,flags", [
    (256, 8, 0, 1), (256, 8, 3, 1), (256, 8, 3, 0), (512, 5, 2, 1), (1024, 4, 0, 3), (64, 1, 0, 1),
    (4096, 2, 1, 1), (2048, 3, 0, 1), (8192, 2, 1, 1),
    (4096, 3, 2, 3), (8192, 2, 0, 3), (2048, 17, 0, 1),  # FP64 screen on the TMA column pass; > 16 planes
])
def test_image_end_to_end(wst, n, n_w, chunk, flags):
    u, v, w, vis = make_case(n=n, n_vis=4000, seed=7 * n + n_w)
    cfg = wst.Config(n=n, fov=0.1, n_w=n_w, w_min=-200.0, w_max=200.0, flags=flags, planes_per_chunk=chunk)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    img = plan.image()
    ref = oracle.image(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis)
    assert_image_parity(img[0].cpu().numpy(), ref, ocfg_for(cfg, -200.0, 200.0))
    unc = plan.image(flags=wst.WST_NO_CORRECTION)
    ref_u = oracle.image(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis, correct=False)
    assert rel_err(unc[0].cpu().numpy(), ref_u) < TOL
    assert plan.stats()["n_chunks"] == (-(-n_w // chunk) if chunk else 1)


@pytest.mark.parametrize("n", [256, 8192])
def test_image_from_pinned_host_buffers_in_place(wst, n):
    """Page-locked host arrays go straight to wst_plan_set_vis and a page-locked host
    image to wst_image: the kernels read and write them in place.  The image matches the
    oracle and the image computed from device copies of the same arrays."""
    u, v, w, vis = make_case(n=n, n_vis=4000, seed=31 + n)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    plan = wst.Plan(cfg)
    plan.set_vis(pin(u), pin(v), pin(w), pin(vis))
    host_img = torch.empty((1, n, n), dtype=torch.complex64).pin_memory()
    plan.image(out=host_img)
    torch.cuda.synchronize()
    assert plan.stats()["n_kept"] == int((oracle.locate(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis)[3] == 0).sum())
    ref = oracle.image(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis)
    assert_image_parity(host_img[0].numpy(), ref, ocfg_for(cfg, -200.0, 200.0))
    # uncorrected images (the correction amplifies rounding at the corners): the two
    # differ only by the order of the float atomics
    plan.image(out=host_img, flags=wst.WST_NO_CORRECTION)
    torch.cuda.synchronize()
    dev_img = gpu_plan(wst, cfg, u, v, w, vis).image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    assert rel_err(host_img[0].numpy(), dev_img) < 1e-6


def test_set_vis_without_or_with_a_short_workspace_is_oom(wst):
    """WST_ERR_OOM (2) from the host-side check, before any launch, when no workspace is
    set or it is one alignment unit smaller than wst_plan_workspace_bytes asks for; the
    exact size is accepted (a view of a larger buffer, so nothing past it is unmapped)."""
    u, v, w, vis = make_case(n=256, n_vis=1000, seed=5)
    cfg = wst.Config(n=256, fov=0.1, n_w=2, w_min=-200.0, w_max=200.0)
    plan = wst.Plan(cfg)
    args = (dev(u), dev(v), dev(w), dev(vis))
    with pytest.raises(wst.WstError) as e:
        wst.wst_plan_set_vis(plan.handle, *args)
    assert e.value.status == 2
    need = wst.wst_plan_workspace_bytes(plan.handle, u.size)
    buf = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
    wst.wst_plan_set_workspace(plan.handle, buf[:need - 256])
    with pytest.raises(wst.WstError) as e:
        wst.wst_plan_set_vis(plan.handle, *args)
    assert e.value.status == 2
    wst.wst_plan_set_workspace(plan.handle, buf[:need])
    wst.wst_plan_set_vis(plan.handle, *args)
    assert plan.stats()["n_kept"] == u.size


def test_pageable_or_foreign_host_tensors_rejected_by_binding(wst):
    with pytest.raises(ValueError):
        wst._ptr(torch.zeros(4), True)  # not page-locked
    with pytest.raises(ValueError):
        wst._ptr(torch.zeros(4).pin_memory())  # host memory where only device memory is accepted


def rows_case(n, seed, n_dumps=3, n_stations=24, n_chan=8, partial=5):
    """Earth-rotation tracks by row and channel, baselines reaching about 0.8 of the grid's
    half-width at the top channel, the last row partial; random values and weights."""
    rng = np.random.default_rng(seed)
    freqs = np.linspace(120e6, 168e6, n_chan)
    rows, scale = synth.array_rows(n_stations, 0.7 * n / 0.1, n_dumps, freqs, rng)
    n_vis = rows.shape[0] * n_chan - partial
    vis = synth.random_visibilities(n_vis, rng)
    weight = rng.uniform(0.5, 2.0, n_vis).astype(np.float32)
    return rows, scale, vis, weight


def cells(wst, plan, n_vis):
    k = torch.empty(n_vis, dtype=torch.int32, device="cuda")
    i0, j0 = torch.empty_like(k), torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    return k.cpu().numpy(), i0.cpu().numpy(), j0.cpu().numpy()


@pytest.mark.parametrize("n", [256, 8192])
def test_set_vis_rows_placement_and_image(wst, n):
    """wst_plan_set_vis_rows: the coordinates formed in the sort (FP64 product of the
    row's metres and the channel's nu / c, one rounding) place every visibility where the
    oracle's expansion does, the w range from the data included, and the image (weights,
    a partial last row) matches the oracle."""
    rows, scale, vis, weight = rows_case(n, seed=51 + n)
    u, v, w = oracle.expand_rows(rows, scale, vis.size)
    cfg = wst.Config(n=n, fov=0.1, n_w=4, flags=wst.WST_FLAG_KAHAN)  # w range from the data
    plan = wst.Plan(cfg)
    plan.set_vis_rows(dev(rows), dev(scale), dev(vis), dev(weight))
    lo, hi = oracle.resolve_w_range(w, 0.0, 0.0)
    st_ = plan.stats()
    assert st_["w_min"] == lo and st_["w_max"] == hi
    oc = ocfg_for(cfg, lo, hi)
    ko, io, jo, status = oracle.locate(oc, u, v, w, vis, weight)
    k, i0, j0 = cells(wst, plan, vis.size)
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(i0, io)
    np.testing.assert_array_equal(j0, jo)
    assert st_["n_kept"] == int((status == 0).sum()) > 0.9 * vis.size
    img = plan.image()
    assert_image_parity(img[0].cpu().numpy(), oracle.image(oc, u, v, w, vis, weight), oc)


def test_set_vis_rows_pinned_host_and_batched(wst):
    """Rows, scales, values and weights in page-locked host memory, two images split by
    batch offsets: the images equal those of wst_plan_set_vis on device copies of the
    expanded coordinates (uncorrected; up to the order of float atomics)."""
    rows, scale, vis, weight = rows_case(256, seed=61, n_dumps=4)
    u, v, w = oracle.expand_rows(rows, scale, vis.size)
    off = [0, vis.size // 3, vis.size]
    cfg = wst.Config(n=256, fov=0.1, n_w=3, batch=2)  # per-image w ranges from the data
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    plan = wst.Plan(cfg)
    plan.set_vis_rows(pin(rows), pin(scale), pin(vis), pin(weight), off)
    host_img = torch.empty((2, 256, 256), dtype=torch.complex64).pin_memory()
    plan.image(out=host_img, flags=wst.WST_NO_CORRECTION)
    torch.cuda.synchronize()
    k, i0, j0 = cells(wst, plan, vis.size)
    ref_plan = gpu_plan(wst, cfg, u, v, w, vis, weight, off)
    kr, ir, jr = cells(wst, ref_plan, vis.size)
    np.testing.assert_array_equal(k, kr)
    np.testing.assert_array_equal(i0, ir)
    np.testing.assert_array_equal(j0, jr)
    ref = ref_plan.image(flags=wst.WST_NO_CORRECTION).cpu().numpy()
    for b in range(2):
        assert rel_err(host_img[b].numpy(), ref[b]) < 1e-6


def test_set_vis_rows_rejects_bad_arguments(wst):
    cfg = wst.Config(n=256, fov=0.1, n_w=2, w_min=-200.0, w_max=200.0)
    plan = wst.Plan(cfg)
    rows = dev(np.zeros((2, 3)))
    vis = dev(np.zeros(7, np.complex64))
    with pytest.raises(wst.WstError):  # 7 visibilities > 2 rows x 3 channels
        plan.set_vis_rows(rows, dev(np.ones(3)), vis)
    with pytest.raises(wst.WstError):  # no channels
        plan.set_vis_rows(rows, dev(np.ones(0)), dev(np.zeros(1, np.complex64)))
    with pytest.raises(ValueError):  # pageable host rows
        plan.set_vis_rows(torch.zeros((2, 3), dtype=torch.float64), dev(np.ones(3)), vis[:6])
    plan.set_vis_rows(rows, dev(np.ones(3)), vis[:6])  # exactly full rows
    assert plan.stats()["n_kept"] == 6


@pytest.mark.parametrize("n", [256, 8192])
def test_wfold_placement_and_image(wst, n):
    """WST_FLAG_WFOLD: w < 0 visibilities are mirrored before placement (the w range from
    the data becomes [min |w|, max |w|]); placement is bit-exact and the image matches the
    oracle run on the mirrored visibilities (its real part is the unfolded dirty image's)."""
    u, v, w, vis = make_case(n=n, n_vis=5000, seed=41 + n)
    cfg = wst.Config(n=n, fov=0.1, n_w=4, flags=wst.WST_FLAG_KAHAN | wst.WST_FLAG_WFOLD)  # range from data
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    fu, fv, fw, fvis = oracle.fold_w(u, v, w, vis)
    lo, hi = oracle.resolve_w_range(fw, 0.0, 0.0)
    st_ = plan.stats()
    assert st_["w_min"] == lo and st_["w_max"] == hi and lo >= 0.0
    k = torch.empty(u.size, dtype=torch.int32, device="cuda")
    i0, j0 = torch.empty_like(k), torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    oc = ocfg_for(cfg, lo, hi)
    ko, io, jo, _ = oracle.locate(oc, fu, fv, fw, fvis)
    np.testing.assert_array_equal(k.cpu().numpy(), ko)
    np.testing.assert_array_equal(i0.cpu().numpy(), io)
    np.testing.assert_array_equal(j0.cpu().numpy(), jo)
    img = plan.image()
    assert_image_parity(img[0].cpu().numpy(), oracle.image(oc, fu, fv, fw, fvis), oc)
    unc = plan.image(flags=wst.WST_NO_CORRECTION)
    assert rel_err(unc[0].cpu().numpy(), oracle.image(oc, fu, fv, fw, fvis, correct=False)) < TOL
    with pytest.raises(wst.WstError):
        plan.degrid(img)


@pytest.mark.parametrize("n,chunk", [(256, 0), (256, 2), (4096, 0)])
def test_oversampled_grid_image(wst, n, chunk):
    """oversample = 2: a 2N grid of 1/(2 fov) cells and the central N x N of its transform
    (the same pixels); the image matches the oracle's oversampled image (whole image at
    1e-5 of the peak: no corner amplification, the correction stays within the half
    band), also with the planes in chunks (Kahan merge into an N x N image)."""
    u, v, w, vis = make_case(n=n, n_vis=4000, seed=51 + n + chunk)
    cfg = wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0, oversample=2, planes_per_chunk=chunk)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    img = plan.image()
    assert img.shape == (1, n, n)
    oc = ocfg_for(cfg, -200.0, 200.0)
    ref = oracle.image_oversampled(oc, 2, u, v, w, vis)
    assert rel_err(img[0].cpu().numpy(), ref) < TOL
    unc = plan.image(flags=wst.WST_NO_CORRECTION)
    assert rel_err(unc[0].cpu().numpy(), oracle.image_oversampled(oc, 2, u, v, w, vis, correct=False)) < TOL
    # the adjoint of the same plan (the image zero-padded into the grid)
    y = img[0].cpu().numpy()
    got = plan.degrid(img).cpu().numpy()
    assert rel_err(got, oracle.degrid_oversampled(oc, 2, u, v, w, vis, y)) < TOL


def test_oversampled_grid_staged_path(wst):
    """wst_grid returns the 2N x 2N planes; wst_fft_correct adds the central N x N of their
    screened transforms and wst_correct applies the grid's correction to it."""
    n = 256
    u, v, w, vis = make_case(n=n, n_vis=3000, seed=57)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, oversample=2)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    g = torch.empty((3, 2 * n, 2 * n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 3, g)
    oc = ocfg_for(cfg, -200.0, 200.0)
    big = OracleConfig(2 * n, 0.2, 3, -200.0, 200.0, oc.support, oc.kernel, oc.kparam)
    assert rel_err(g.cpu().numpy(), oracle.grid(big, u, v, w, vis)) < TOL
    img = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_fft_correct(plan.handle, 0, 3, g, img)
    assert rel_err(img[0].cpu().numpy(), oracle.image_oversampled(oc, 2, u, v, w, vis, correct=False)) < TOL
    wst.wst_correct(plan.handle, img)
    assert rel_err(img[0].cpu().numpy(), oracle.image_oversampled(oc, 2, u, v, w, vis)) < TOL


@pytest.mark.parametrize("kernel,W,param", [("es", 8, 2.3 * 8), ("gauss", 8, 0.925), ("table", 8, None)])
def test_image_kernels(wst, kernel, W, param):
    n = 256
    u, v, w, vis = make_case(n=n, n_vis=3000, seed=11)
    table = None
    if kernel == "table":
        x = np.linspace(-W / 2, W / 2, W * 64 + 1)
        table = np.exp(-x**2 / (2 * 0.925**2)) * (1 + 0.1 * np.cos(3 * x))
    kid = {"gauss": 0, "es": 1, "table": 2}[kernel]
    cfg = wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0, support=W, kernel=kid,
                     kparam=param or 0.0, ktable_len=0 if table is None else table.size)
    plan = gpu_plan(wst, cfg, u, v, w, vis, table=table)
    img = plan.image()
    t32 = None if table is None else table.astype(np.float32)
    oc = ocfg_for(cfg, -200.0, 200.0, t32)
    ref = oracle.image(oc, u, v, w, vis)
    assert_image_parity(img[0].cpu().numpy(), ref, oc)
    # the grid-correction table itself, read back through wst_correct on ones
    ones = torch.ones((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_correct(plan.handle, ones)
    cc = np.outer(correction(oc), correction(oc))
    assert np.abs(ones[0].cpu().numpy().real / cc - 1).max() < 1e-6


def test_image_weights_and_nonfinite(wst):
    n = 256
    u, v, w, vis = make_case(n=n, n_vis=3000, seed=5)
    wt = np.random.default_rng(9).uniform(0.0, 3.0, u.size).astype(np.float32)
    wt[10] = np.inf
    w[11] = np.nan
    cfg = wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0)
    plan = gpu_plan(wst, cfg, u, v, w, vis, weight=wt)
    img = plan.image()
    ref = oracle.image(ocfg_for(cfg, -200.0, 200.0), u, v, w, vis, wt)
    assert_image_parity(img[0].cpu().numpy(), ref, ocfg_for(cfg, -200.0, 200.0))
    assert plan.stats()["n_nonfinite"] == 2


def test_image_empty_and_all_dropped(wst):
    n = 128
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-1.0, w_max=1.0)
    plan = wst.Plan(cfg)
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    plan.set_vis(e, e, e, torch.empty(0, dtype=torch.complex64, device="cuda"))
    img = plan.image()
    assert torch.count_nonzero(img).item() == 0
    far = np.full(100, 5000.0, np.float32)
    plan.set_vis(dev(far), dev(far), dev(np.zeros(100, np.float32)), dev(np.ones(100, np.complex64)))
    img = plan.image()
    assert torch.count_nonzero(img).item() == 0
    assert plan.stats()["n_dropped"] == 100


def test_single_visibility_flat_image(wst):
    n = 256
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-30.0, w_max=30.0)
    plan = gpu_plan(wst, cfg, np.zeros(1, np.float32), np.zeros(1, np.float32), np.zeros(1, np.float32),
                    np.ones(1, np.complex64))
    img = plan.image()[0].cpu().numpy()
    ref = oracle.image(ocfg_for(cfg, -30.0, 30.0), [0.0], [0.0], [0.0], np.ones(1, np.complex64))
    assert_image_parity(img, ref, ocfg_for(cfg, -30.0, 30.0))
    c = slice(n // 4, 3 * n // 4)
    assert np.abs(img[c, c] - 1).max() < 3e-3


def test_batched_images(wst):
    n, n_w = 256, 4
    counts = [500, 0, 2500, 1200]
    rng = np.random.default_rng(17)
    us, vs, ws, viss = [], [], [], []
    for c in counts:
        u, v, w = synth.disk_uvw(c, 0.45 * n / 0.1, 150.0, rng)
        us.append(u); vs.append(v); ws.append(w); viss.append(synth.random_visibilities(c, rng))
    off = np.concatenate([[0], np.cumsum(counts)])
    U, V, Wv, VIS = (np.concatenate(x) for x in (us, vs, ws, viss))
    cfg = wst.Config(n=n, fov=0.1, n_w=n_w, batch=len(counts), planes_per_chunk=3)
    plan = gpu_plan(wst, cfg, U, V, Wv, VIS, offsets=off)
    img = plan.image().cpu().numpy()
    for b, c in enumerate(counts):
        if c == 0:
            assert np.all(img[b] == 0)
            continue
        lo, hi = oracle.resolve_w_range(ws[b], 0.0, 0.0)
        ref = oracle.image(ocfg_for(cfg, lo, hi), us[b], vs[b], ws[b], viss[b])
        assert_image_parity(img[b], ref, ocfg_for(cfg, lo, hi))


def test_wide_field_outside_sphere_zero(wst):
    n = 128
    cfg = wst.Config(n=n, fov=2.4, n_w=2, w_min=-5.0, w_max=5.0)
    u, v, w, vis = make_case(n=n, fov=2.4, n_vis=500, w_half=5.0)
    plan = gpu_plan(wst, cfg, u, v, w, vis)
    img = plan.image()[0].cpu().numpy()
    ref = oracle.image(ocfg_for(cfg, -5.0, 5.0), u, v, w, vis)
    assert_image_parity(img, ref, ocfg_for(cfg, -5.0, 5.0))
    assert np.all(img[ref == 0] == 0)
