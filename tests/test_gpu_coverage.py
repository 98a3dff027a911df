"""GPU parity for the configurations the benchmark reports numbers for, at their sizes.

* W = 8 kernels (Gaussian sigma = 0.925, the trained table and the Kaiser-Bessel and
  prolate spheroidal tables) on the fixed-point rows of images of 8192^2 and up: the
  full image at 8192^2 against ``oracle.image``, and 16384^2 at sampled pixels against
  ``oracle.image_pixels``;
* the staged row FFT of a 16384-point grid (``wst_fft_correct``, the TMA-prefetched
  row kernel);
* the batched workload at its real shape (64 images of 2048^2, 16 planes, 37.7M
  visibilities of uneven counts, one launch per stage), several images checked;
* placement of w on, and 1-2 FP32 steps from, plane boundaries, bit for bit.

Tolerance: 1e-5 of the peak (the image before the grid correction everywhere, the
corrected image on the central half; over the full corrected image the FP32 budget of
``test_gpu_parity.assert_image_parity``).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import OracleConfig
from paper_2301_06061_gb300 import kernels, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    ref = np.asarray(ref)
    return float(np.abs(np.asarray(gpu, dtype=np.complex128) - ref).max() / np.abs(ref).max())


def correction(ocfg):
    n = ocfg.n
    return 1.0 / oracle.kernel_ft(ocfg, (np.arange(n) - n // 2) / n)


def assert_image_parity(gpu, ref, ocfg, tol=TOL):
    gpu = np.asarray(gpu, dtype=np.complex128)
    n = ref.shape[-1]
    cc = np.outer(correction(ocfg), correction(ocfg))
    u_peak = np.abs(ref / cc).max()
    err = np.abs(gpu - ref)
    c = slice(n // 4, 3 * n // 4)
    assert err[c, c].max() <= tol * np.abs(ref[c, c]).max(), err[c, c].max() / np.abs(ref[c, c]).max()
    budget = tol * u_peak * cc + 1e-6 * np.abs(ref)
    assert np.all(err <= budget), float((err / budget).max())


def learned_table():
    from paper_2301_06061_gb300 import learned

    return learned.load_table(os.path.join(ROOT, "paper_2301_06061_gb300", "data", "learned_kernel_w8.npz"))


def w8_kernel(wst, name):
    """(wst.Config kwargs, oracle kernel args, device table or None) of a W = 8 kernel:
    the Gaussian, the trained table, or the Kaiser-Bessel / prolate spheroidal window
    tabulated for a grid the size of the image (oversampling 1)."""
    if name == "gauss8":
        return dict(support=8, kparam=0.925), ("gauss", 0.925, None), None
    if name == "kb8":
        tab = kernels.kaiser_bessel_table(8, kernels.kaiser_bessel_beta(8, 1.0))
    elif name == "pswf8":
        tab = kernels.pswf_table(8, kernels.pswf_c(8, 1.0))
    else:
        tab = learned_table()
    tab = tab.astype(np.float32)
    return (dict(support=8, kernel=wst.WST_KERNEL_TABLE, kparam=0.0, ktable_len=int(tab.size)),
            ("table", 0.0, tab.astype(np.float64)), dev(tab))


def sample_pixels(n, count, seed):
    rng = np.random.default_rng(seed)
    pa = rng.integers(0, n, count)
    pb = rng.integers(0, n, count)
    extra_a = np.array([n // 2, 0, n - 1, 0, n - 1, n // 2, 0, n - 1])
    extra_b = np.array([n // 2, 0, 0, n - 1, n - 1, 0, n // 2, n // 2])
    return np.concatenate([pa, extra_a]).astype(np.int32), np.concatenate([pb, extra_b]).astype(np.int32)


def dense_tracks(n_vis, seed):
    """Core-dense earth-rotation tracks of the benchmark's array (300 stations, 64
    channels), three dumps over 8 h, ``n_vis`` of them drawn at random."""
    work = synth.large(n_vis=3 * 300 * 299 // 2 * 64)
    sel = np.sort(np.random.default_rng(seed).choice(work.n_vis, n_vis, replace=False))
    return work.u[sel], work.v[sel], work.w[sel]


# ------------------------------------------------------------------------------------------
# W = 8 on fixed-point rows
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", ["gauss8", "learned", "kb8", "pswf8"])
def test_w8_fixed_point_rows_full_image_8192(wst, kernel):
    """The array workload's tracks (60 stations, 16 channels, 4.08M visibilities,
    core-dense) on an 8192^2 grid of FoV 0.2 (every row in the fixed-point path), 4
    planes; the whole image against the FP64 oracle, corrected and not."""
    work = synth.array()
    vis = synth.random_visibilities(work.n_vis, np.random.default_rng(81))
    n, fov, n_w = 8192, 0.2, 4
    kw, (okind, oparam, otab), table = w8_kernel(wst, kernel)
    plan = wst.Plan(wst.Config(n=n, fov=fov, n_w=n_w, **kw))
    if table is not None:
        plan.set_kernel_table(table)
    plan.set_vis(dev(work.u), dev(work.v), dev(work.w), dev(vis))
    img_u = plan.image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    img_c = plan.image()[0].cpu().numpy()
    st = plan.stats()
    assert st["n_kept"] == work.n_vis and st["device_error"] == 0
    lo, hi = oracle.resolve_w_range(work.w, 0.0, 0.0)
    ocfg = OracleConfig(n, fov, n_w, lo, hi, 8, okind, oparam, otab)
    ref_u = oracle.image(ocfg, work.u, work.v, work.w, vis, correct=False)
    assert rel_err(img_u, ref_u) < TOL
    del ref_u
    ref_c = oracle.image(ocfg, work.u, work.v, work.w, vis)
    assert_image_parity(img_c, ref_c, ocfg)


@pytest.mark.parametrize("kernel", ["gauss8", "learned", "kb8", "pswf8"])
def test_w8_kernels_16384_sampled(wst, kernel):
    """16384^2, FoV 0.5 (the benchmark's geometry and fixed-point rows), 4 planes in 2
    chunks, 1.5M core-dense visibilities; 264 pixels against the oracle's pixel-wise
    evaluation."""
    u, v, w = dense_tracks(1_500_000, 82)
    vis = synth.random_visibilities(u.size, np.random.default_rng(83))
    n, fov, n_w = 16384, 0.5, 4
    kw, (okind, oparam, otab), table = w8_kernel(wst, kernel)
    plan = wst.Plan(wst.Config(n=n, fov=fov, n_w=n_w, planes_per_chunk=2, **kw))
    if table is not None:
        plan.set_kernel_table(table)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    pa, pb = sample_pixels(n, 256, 84)
    ia, ib = dev(pa).long(), dev(pb).long()
    got_u = plan.image(flags=wst.WST_NO_CORRECTION)[0][ib, ia].cpu().numpy()
    got_c = plan.image()[0][ib, ia].cpu().numpy()
    lo, hi = oracle.resolve_w_range(w, 0.0, 0.0)
    ocfg = OracleConfig(n, fov, n_w, lo, hi, 8, okind, oparam, otab)
    ref_u = oracle.image_pixels(ocfg, u, v, w, vis, pa, pb, correct=False)
    ref_c = ref_u / (oracle.kernel_ft(ocfg, (pa - n // 2) / n) * oracle.kernel_ft(ocfg, (pb - n // 2) / n))
    assert np.abs(got_u - ref_u).max() <= TOL * np.abs(ref_u).max()
    central = (np.abs(pa - n // 2) < n // 4) & (np.abs(pb - n // 2) < n // 4)
    assert np.abs(got_c - ref_c)[central].max() <= TOL * np.abs(ref_c[central]).max()


# ------------------------------------------------------------------------------------------
# the staged row FFT of a 16384-point grid (TMA-prefetched rows)
# ------------------------------------------------------------------------------------------

def test_fft_correct_staged_16384(wst):
    """wst_grid + wst_fft_correct + wst_correct on a 16384 grid, 2 planes of 5000
    visibilities: the row pass of wst_fft_correct at this size is the TMA-prefetched
    row kernel with bounded waits."""
    rng = np.random.default_rng(85)
    n, fov, n_w = 16384, 0.5, 2
    u, v, w = synth.disk_uvw(5000, 0.45 * n / fov, 300.0, rng)
    vis = synth.random_visibilities(5000, rng)
    plan = wst.Plan(wst.Config(n=n, fov=fov, n_w=n_w, w_min=-300.0, w_max=300.0))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    g = torch.empty((n_w, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, n_w, g)
    img = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_fft_correct(plan.handle, 0, n_w, g, img)
    del g
    pa, pb = sample_pixels(n, 256, 86)
    ia, ib = dev(pa).long(), dev(pb).long()
    got_u = img[0][ib, ia].cpu().numpy()
    wst.wst_correct(plan.handle, img)
    got_c = img[0][ib, ia].cpu().numpy()
    assert plan.stats()["device_error"] == 0
    ocfg = OracleConfig(n, fov, n_w, -300.0, 300.0, 7)
    ref_u = oracle.image_pixels(ocfg, u, v, w, vis, pa, pb, correct=False)
    ref_c = ref_u / (oracle.kernel_ft(ocfg, (pa - n // 2) / n) * oracle.kernel_ft(ocfg, (pb - n // 2) / n))
    assert np.abs(got_u - ref_u).max() <= TOL * np.abs(ref_u).max()
    central = (np.abs(pa - n // 2) < n // 4) & (np.abs(pb - n // 2) < n // 4)
    assert np.abs(got_c - ref_c)[central].max() <= TOL * np.abs(ref_c[central]).max()


# ------------------------------------------------------------------------------------------
# the batched workload at its real shape
# ------------------------------------------------------------------------------------------

def test_batched_workload_real_shape(wst):
    """64 channel images of 2048^2, 16 planes each, counts log-uniform in [1e5, 2e6]
    (37.7M visibilities), all planes resident (the benchmark's launch configuration); the
    smallest, the largest and two other images against the oracle."""
    work = synth.batched()
    vis = synth.random_visibilities(work.n_vis, np.random.default_rng(87))
    off = work.batch_offsets
    batch = off.size - 1
    plan = wst.Plan(wst.Config(n=work.n, fov=work.fov, n_w=work.n_w, batch=batch))
    plan.set_vis(dev(work.u), dev(work.v), dev(work.w), dev(vis), None, [int(x) for x in off])
    img = plan.image()
    st = plan.stats()
    assert st["device_error"] == 0 and st["n_kept"] + st["n_dropped"] == work.n_vis
    counts = np.diff(off)
    picks = sorted({int(np.argmin(counts)), int(np.argmax(counts)), 17, 40})
    for b in picks:
        s = slice(off[b], off[b + 1])
        u, v, w, vv = work.u[s], work.v[s], work.w[s], vis[s]
        lo, hi = oracle.resolve_w_range(w, 0.0, 0.0)
        ocfg = OracleConfig(work.n, work.fov, work.n_w, lo, hi, 7)
        ref = oracle.image(ocfg, u, v, w, vv)
        assert_image_parity(img[b].cpu().numpy(), ref, ocfg)


# ------------------------------------------------------------------------------------------
# placement of w at plane boundaries
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("w_min,w_max,n_w", [
    (-256.0, 256.0, 32), (-200.0, 200.0, 8), (-6547.25, 6728.5, 32), (-1000.0, 2000.0, 3),
    (-3.3333332538604736, 6.6666669845581055, 48),
])
def test_vis_cells_at_plane_boundaries_bit_exact(wst, w_min, w_max, n_w):
    """w on, and 1-2 FP32 steps from, every plane boundary (including exact hits that the
    oracle's rounded scale sends to the lower plane, and the subnormal neighbours of a
    boundary at w = 0): the sort's plane equals the oracle's, with the range given and
    with the range taken from the data (the same end points are in the data)."""
    F = __import__("fractions").Fraction
    ws = []
    for k in range(1, n_w):
        c = np.float32(float(F(w_min) + k * (F(w_max) - F(w_min)) / n_w))
        ws += [c, np.nextafter(c, np.float32(np.inf)), np.nextafter(c, np.float32(-np.inf))]
        ws += [np.nextafter(ws[-2], np.float32(np.inf)), np.nextafter(ws[-1], np.float32(-np.inf))]
    w = np.array(ws + [w_min, w_max], np.float32)
    z = np.zeros(w.size, np.float32)
    vis = np.ones(w.size, np.complex64)
    for cw_min, cw_max in ((w_min, w_max), (0.0, 0.0)):
        plan = wst.Plan(wst.Config(n=64, fov=0.1, n_w=n_w, w_min=cw_min, w_max=cw_max))
        plan.set_vis(dev(z), dev(z), dev(w), dev(vis))
        k = torch.empty(w.size, dtype=torch.int32, device="cuda")
        i0, j0 = torch.empty_like(k), torch.empty_like(k)
        wst.wst_vis_cells(plan.handle, k, i0, j0)
        ko, _, _, _ = oracle.locate(OracleConfig(64, 0.1, n_w, w_min, w_max, 7), z, z, w, vis)
        np.testing.assert_array_equal(k.cpu().numpy(), ko)


# ------------------------------------------------------------------------------------------
# failure detection: a bounded device wait that runs out
# ------------------------------------------------------------------------------------------

def test_row_copy_wait_expiry_reports_timeout_and_plans_stay_usable(wst):
    """With the plan's data-wait limit at 0 every CTA of the 16384-point row FFT gives up
    on its first row copy: the device error word reads WST_ERR_TIMEOUT (each CTA waits,
    with the full limit, for the copy it has in flight before it exits).  The same plan
    after the limit is restored and the visibilities set again, and a fresh plan, both
    run the same call cleanly and agree with the oracle."""
    rng = np.random.default_rng(88)
    n, fov = 16384, 0.5
    u, v, w = synth.disk_uvw(2000, 0.45 * n / fov, 100.0, rng)
    vis = synth.random_visibilities(2000, rng)
    cfg = wst.Config(n=n, fov=fov, n_w=1, w_min=-100.0, w_max=100.0)
    du, dv, dw, dvis = dev(u), dev(v), dev(w), dev(vis)
    g = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    img = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    plan = wst.Plan(cfg)
    plan.set_vis(du, dv, dw, dvis)
    wst.wst_plan_set_wait_limit(plan.handle, 0)
    wst.wst_grid(plan.handle, 0, 1, g)
    wst.wst_fft_correct(plan.handle, 0, 1, g, img)
    st = plan.stats()
    assert st["device_error"] == 4  # WST_ERR_TIMEOUT
    pa, pb = sample_pixels(n, 56, 89)
    ocfg = OracleConfig(n, fov, 1, -100.0, 100.0, 7)
    ref = oracle.image_pixels(ocfg, u, v, w, vis, pa, pb, correct=False)
    ia, ib = dev(pa).long(), dev(pb).long()
    for fresh in (False, True):
        if fresh:
            plan.close()
            plan = wst.Plan(cfg)
        else:
            wst.wst_plan_set_wait_limit(plan.handle, 2_000_000_000)
        plan.set_vis(du, dv, dw, dvis)
        img.zero_()
        wst.wst_grid(plan.handle, 0, 1, g)
        wst.wst_fft_correct(plan.handle, 0, 1, g, img)
        assert plan.stats()["device_error"] == 0
        got = img[0][ib, ia].cpu().numpy()
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


# ------------------------------------------------------------------------------------------
# the transform stage against cuFFT (comparison only: cuFFT is never on the product path)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [4096, 16384])
def test_transform_matches_cufft(wst, n):
    """A gridded plane transformed by this library (wst_fft_correct on a one-plane plan
    whose plane centre is w = 0, so the screen is exactly 1: the centred transform of
    Eq. 2 itself) and by cuFFT (torch.fft, the same convention by centring signs); at
    4096^2 both also against the oracle's FP64 transform of the same plane."""
    import bench

    rng = np.random.default_rng(90 + n)
    fov = 0.5 if n == 16384 else 0.2
    u, v, w = synth.disk_uvw(200_000, 0.45 * n / fov, 1.0, rng)
    vis = synth.random_visibilities(u.size, rng)
    plan = wst.Plan(wst.Config(n=n, fov=fov, n_w=1, w_min=-1.0, w_max=1.0))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    g = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 1, g)
    ref = bench.centred_fft_cufft(torch, g)[0]
    ours = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_fft_correct(plan.handle, 0, 1, g.clone(), ours)
    peak = ref.abs().max().item()
    assert (ours[0] - ref).abs().max().item() <= TOL * peak
    if n == 4096:
        truth = oracle.fft2_centered(g[0].cpu().numpy().astype(np.complex128), +1)
        tp = np.abs(truth).max()
        assert np.abs(ours[0].cpu().numpy() - truth).max() <= TOL * tp
        assert np.abs(ref.cpu().numpy() - truth).max() <= TOL * tp


def test_rows_gridded_counts_the_occupied_rows(wst):
    """wst_stats.n_rows_gridded: the (plane, row) items some visibility's W-row footprint
    reaches (the oracle's placements j0 .. j0 + W - 1 per plane), over all chunks."""
    rng = np.random.default_rng(92)
    n, n_w, W = 1024, 5, 7
    u, v, w = synth.disk_uvw(3000, 0.3 * n / 0.1, 200.0, rng)
    vis = synth.random_visibilities(u.size, rng)
    for chunk in (0, 2):
        plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=n_w, w_min=-200.0, w_max=200.0, planes_per_chunk=chunk))
        plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
        plan.image()
        got = plan.stats()["n_rows_gridded"]
        k, _, j0, st = oracle.locate(OracleConfig(n, 0.1, n_w, -200.0, 200.0, W), u, v, w, vis)
        rows = {(int(kk), int(jj) + d) for kk, jj, ss in zip(k, j0, st) if ss == 0 for d in range(W)}
        assert got == len(rows)
        plan.image_range(1, 3)
        assert plan.stats()["n_rows_gridded"] == len({r for r in rows if 1 <= r[0] < 3})
