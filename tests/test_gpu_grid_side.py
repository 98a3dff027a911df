"""GPU parity of an explicit grid side (``wst_config.grid_n``): an image of N pixels (N
even, not a power of two) cropped from the transform of a grid of M cells (a power of
two), oversampling factor M/N between 1 and 2, against the oracle's ``image_on_grid``,
``degrid_on_grid`` and ``kernel_grad_on_grid``.  The crop starts at grid column
(M - N)/2, which is not a multiple of the 16-column bands of column stage B: the bands at
both image edges are partial.

Tolerance: 1e-5 of the peak for the uncorrected image and the adjoint; the corrected
image within the FP32 budget |dD| <= 1e-5 max|U| C_a C_b + 1e-6 |D|, C = 1/Ghat at the
image's frequencies (a - N/2)/M (up to ~10 per axis at M/N = 1.25 for the Gaussian
W = 7), and at 1e-5 of the peak on the central half.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(gpu, ref):
    ref = np.asarray(ref)
    return float(np.abs(np.asarray(gpu, np.complex128) - ref).max() / max(np.abs(ref).max(), 1e-300))


def corr_axis(ocfg, m, idx):
    """1/Ghat at image pixels idx of an image cropped from an m-cell grid."""
    n = ocfg.n
    return 1.0 / oracle.kernel_ft(oracle.grid_config(ocfg, m), (np.asarray(idx) - n // 2) / m)


def assert_corrected(gpu, ref, ocfg, m):
    gpu = np.asarray(gpu, np.complex128)
    n = ocfg.n
    cc = np.outer(corr_axis(ocfg, m, np.arange(n)), corr_axis(ocfg, m, np.arange(n)))
    err = np.abs(gpu - ref)
    c = slice(n // 4, 3 * n // 4)
    assert err[c, c].max() <= TOL * np.abs(ref[c, c]).max()
    budget = TOL * np.abs(ref / cc).max() * cc + 1e-6 * np.abs(ref)
    assert np.all(err <= budget), float((err / budget).max())


def case(n, n_vis, seed, fov=0.1):
    rng = np.random.default_rng(seed)
    u, v, w = synth.disk_uvw(n_vis, 0.45 * n / fov, 200.0, rng)
    vis = synth.random_visibilities(n_vis, rng)
    return u, v, w, vis, rng


@pytest.mark.parametrize("n,m,chunk", [(204, 256, 0), (170, 256, 2), (3276, 4096, 0)])
def test_image_and_adjoint_on_a_grid_of_side_m(wst, n, m, chunk):
    u, v, w, vis, rng = case(n, 4000, 61 + n + chunk)
    cfg = wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0, grid_n=m, planes_per_chunk=chunk)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    st = plan.stats()
    assert st["n_kept"] == u.size
    oc = OracleConfig(n, 0.1, 4, -200.0, 200.0, 7)
    # placement on the grid is the oracle's, bit for bit
    k = torch.empty(u.size, dtype=torch.int32, device="cuda")
    i0 = torch.empty_like(k)
    j0 = torch.empty_like(k)
    wst.wst_vis_cells(plan.handle, k, i0, j0)
    ko, io, jo, _ = oracle.locate(oracle.grid_config(oc, m), u, v, w, vis)
    np.testing.assert_array_equal(k.cpu().numpy(), ko)
    np.testing.assert_array_equal(i0.cpu().numpy(), io)
    np.testing.assert_array_equal(j0.cpu().numpy(), jo)
    img = plan.image()
    assert img.shape == (1, n, n)
    assert_corrected(img[0].cpu().numpy(), oracle.image_on_grid(oc, m, u, v, w, vis), oc, m)
    unc = plan.image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    assert rel_err(unc, oracle.image_on_grid(oc, m, u, v, w, vis, correct=False)) < TOL
    y = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    for flags, corr in ((0, True), (wst.WST_NO_CORRECTION, False)):
        got = plan.degrid(dev(y[None]), flags=flags).cpu().numpy()
        assert rel_err(got, oracle.degrid_on_grid(oc, m, u, v, w, vis, y, correct=corr)) < TOL


def test_staged_path_on_a_grid_of_side_m(wst):
    """wst_grid returns the M x M planes; wst_fft_correct adds the central N x N of their
    screened transforms and wst_correct applies the grid's correction to it."""
    n, m = 204, 256
    u, v, w, vis, _ = case(n, 3000, 67)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, grid_n=m)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    g = torch.empty((3, m, m), dtype=torch.complex64, device="cuda")
    wst.wst_grid(plan.handle, 0, 3, g)
    oc = OracleConfig(n, 0.1, 3, -200.0, 200.0, 7)
    assert rel_err(g.cpu().numpy(), oracle.grid(oracle.grid_config(oc, m), u, v, w, vis)) < TOL
    img = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    wst.wst_fft_correct(plan.handle, 0, 3, g, img)
    assert rel_err(img[0].cpu().numpy(), oracle.image_on_grid(oc, m, u, v, w, vis, correct=False)) < TOL
    wst.wst_correct(plan.handle, img)
    assert_corrected(img[0].cpu().numpy(), oracle.image_on_grid(oc, m, u, v, w, vis), oc, m)


def test_table_kernel_and_its_gradient_on_a_grid_of_side_m(wst):
    n, m, W = 204, 256, 8
    L = W * 64 + 1
    tab = np.exp(-np.linspace(-W / 2, W / 2, L) ** 2 / (2 * 0.925**2))
    u, v, w, vis, rng = case(n, 3000, 71)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, support=W, kernel=wst.WST_KERNEL_TABLE,
                     ktable_len=L, kparam=0.0, grid_n=m)
    plan = wst.Plan(cfg)
    plan.set_kernel_table(dev(tab.astype(np.float32)))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    oc = OracleConfig(n, 0.1, 3, -200.0, 200.0, W, "table", 0.0, tab.astype(np.float32).astype(np.float64))
    img = plan.image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    assert rel_err(img, oracle.image_on_grid(oc, m, u, v, w, vis, correct=False)) < TOL
    dU = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    got = plan.kernel_grad(dev(dU[None])).cpu().numpy()
    ref = oracle.kernel_grad_on_grid(oc, m, u, v, w, vis, dU)
    # a sum over the image of products with a random dimage: the FP32 rounding of the
    # transform shows through its cancellation (1e-4 of the peak, as on the plain grid)
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


def test_16384_grid_image_of_13108_pixels_sampled(wst):
    """M = 16384 (the TMA-fed column stage B and the fixed-point rows), N = 13108
    (M/N = 1.25; the crop starts 6 columns into a band): sampled pixels, edges included,
    against the oracle evaluated pixel by pixel on the grid."""
    n, m = 13108, 16384
    u, v, w, vis, rng = case(n, 20000, 73)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, grid_n=m)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    img_u = plan.image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    img_c = plan.image()[0].cpu().numpy()
    pa = np.concatenate([rng.integers(0, n, 120), [0, n - 1, 0, n - 1, n // 2, 1, n - 2, 9, 10]]).astype(np.int32)
    pb = np.concatenate([rng.integers(0, n, 120), [0, 0, n - 1, n - 1, n // 2, n - 2, 1, 3, n - 11]]).astype(np.int32)
    oc = OracleConfig(n, 0.1, 3, -200.0, 200.0, 7)
    c = (m - n) // 2
    ref_u = oracle.image_pixels(oracle.grid_config(oc, m), u, v, w, vis, pa + c, pb + c, correct=False)
    got_u = img_u[pb, pa].astype(np.complex128)
    assert np.abs(got_u - ref_u).max() <= TOL * np.abs(ref_u).max()
    ref_c = ref_u * corr_axis(oc, m, pa) * corr_axis(oc, m, pb)
    got_c = img_c[pb, pa].astype(np.complex128)
    central = (np.abs(pa - n // 2) < n // 4) & (np.abs(pb - n // 2) < n // 4)
    assert np.abs(got_c - ref_c)[central].max() <= TOL * np.abs(ref_c[central]).max()
    # every pixel: the budget of the corrected image (FP32 rounding times the correction)
    cc = corr_axis(oc, m, pa) * corr_axis(oc, m, pb)
    assert np.all(np.abs(got_c - ref_c) <= TOL * np.abs(ref_u).max() * cc + 1e-6 * np.abs(ref_c))
