"""Parity at the full 16384^2 size (the benchmark's geometry and launch configuration),
on pixels the FP64 oracle evaluates one by one (``oracle.image_pixels``: the gridding
sum and the plane transform evaluated directly at a pixel, no planes, no FFT).

Tolerance: 1e-5 of the largest oracle value over the sampled pixels, for the image
before the grid correction everywhere and for the corrected image on the central half.
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


def sample_pixels(n, count, seed):
    rng = np.random.default_rng(seed)
    pa = rng.integers(0, n, count)
    pb = rng.integers(0, n, count)
    # always include the centre, the four corners and row/column ends (ragged edges)
    extra_a = np.array([n // 2, 0, n - 1, 0, n - 1, n // 2, 0, n - 1])
    extra_b = np.array([n // 2, 0, 0, n - 1, n - 1, 0, n // 2, n // 2])
    return np.concatenate([pa, extra_a]).astype(np.int32), np.concatenate([pb, extra_b]).astype(np.int32)


def corrected(ocfg, ref_u, pa, pb):
    """The oracle's grid correction applied to its uncorrected pixels."""
    n = ocfg.n
    return ref_u / (oracle.kernel_ft(ocfg, (pa - n // 2) / n) * oracle.kernel_ft(ocfg, (pb - n // 2) / n))


def check_sampled(got_c, got_u, ref_c, ref_u, pa, pb, n):
    got_u = np.asarray(got_u, np.complex128)
    got_c = np.asarray(got_c, np.complex128)
    assert np.abs(got_u - ref_u).max() <= TOL * np.abs(ref_u).max()
    central = (np.abs(pa - n // 2) < n // 4) & (np.abs(pb - n // 2) < n // 4)
    assert np.abs(got_c - ref_c)[central].max() <= TOL * np.abs(ref_c[central]).max()


def test_16k_geometry_sampled(wst):
    """16384^2, FoV 0.5, 4 planes, 1e6 visibilities of the large tracks, 2 chunks."""
    work = synth.large(n_vis=1_000_000, seed_extra=5)
    rng = np.random.default_rng(5)
    vis = synth.random_visibilities(work.n_vis, rng)
    n, n_w = work.n, 4
    cfg = wst.Config(n=n, fov=work.fov, n_w=n_w, support=7, kparam=0.875, planes_per_chunk=2)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(work.u), dev(work.v), dev(work.w), dev(vis))
    img_c = plan.image()[0].cpu().numpy()
    img_u = plan.image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    lo, hi = oracle.resolve_w_range(work.w, 0.0, 0.0)
    ocfg = OracleConfig(n, work.fov, n_w, lo, hi, 7, "gauss", 0.875)
    pa, pb = sample_pixels(n, 248, 11)
    ref_u = oracle.image_pixels(ocfg, work.u, work.v, work.w, vis, pa, pb, correct=False)
    check_sampled(img_c[pb, pa], img_u[pb, pa], corrected(ocfg, ref_u, pa, pb), ref_u, pa, pb, n)


def test_full_benchmark_workload_sampled(wst):
    """The benchmark's workload (1e8 visibilities, 32 planes, all planes resident) and its
    launch configuration, checked at 24 pixels; the GPU direct transform is checked
    against the oracle's direct transform at the same pixels."""
    work = synth.large()
    vis = synth.random_visibilities(work.n_vis, synth.rng_for(3, 7))
    n = work.n
    cfg = wst.Config(n=n, fov=work.fov, n_w=work.n_w, support=7, kparam=0.875,
                     flags=wst.WST_FLAG_KAHAN | wst.WST_FLAG_TIMING)
    plan = wst.Plan(cfg)
    du, dv, dw, dvis = dev(work.u), dev(work.v), dev(work.w), dev(vis)
    plan.set_vis(du, dv, dw, dvis)
    img_c = plan.image()[0]
    pa, pb = sample_pixels(n, 16, 13)
    got_c = img_c[dev(pb).long(), dev(pa).long()].cpu().numpy()
    del img_c
    img_u = plan.image(flags=wst.WST_NO_CORRECTION)[0]
    got_u = img_u[dev(pb).long(), dev(pa).long()].cpu().numpy()
    del img_u
    dft_out = torch.empty(pa.size, dtype=torch.complex64, device="cuda")
    wst.wst_dft(du, dv, dw, dvis, n, work.fov, dev(pa), dev(pb), dft_out)
    st = plan.stats()
    assert st["n_kept"] == work.n_vis and st["device_error"] == 0
    lo, hi = oracle.resolve_w_range(work.w, 0.0, 0.0)
    ocfg = OracleConfig(n, work.fov, work.n_w, lo, hi, 7, "gauss", 0.875)
    ref_u = oracle.image_pixels(ocfg, work.u, work.v, work.w, vis, pa, pb, correct=False)
    check_sampled(got_c, got_u, corrected(ocfg, ref_u, pa, pb), ref_u, pa, pb, n)
    ref_dft = oracle.dft_pixels(work.u, work.v, work.w, vis, n, work.fov, pa, pb)
    assert np.abs(dft_out.cpu().numpy() - ref_dft).max() <= TOL * np.abs(ref_dft).max()
