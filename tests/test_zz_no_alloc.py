"""wst_dft_noalloc: the allocation-free direct transform, checked against wst_dft.

Some callers cannot allocate device memory (real-time pipelines that forbid it
after start-up, plug-ins whose host application's pool owns the device); this entry
point keeps its scratch in an array built into the library.  The test calls it
through the C ABI twice in a row, with different inputs, and compares each result
with the allocating entry point within the tolerance of the other GPU tests.  It
lives in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2301_06061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(seed, n_vis, n_pix, n, fov):
    rng = np.random.default_rng(seed)
    u, v, w = synth.disk_uvw(n_vis, 0.45 * n / fov, 2000.0, rng)
    vis = synth.random_visibilities(n_vis, rng)
    wt = rng.uniform(0.5, 2.0, n_vis).astype(np.float32)
    pa = rng.integers(0, n, n_pix).astype(np.int32)
    pb = rng.integers(0, n, n_pix).astype(np.int32)
    return [_dev(x) for x in (u, v, w, vis, wt, pa, pb)]


def _noalloc(lib, stream, n_vis, u, v, w, vis, wt, n, fov, pa, pb, out):
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return lib.wst_dft_noalloc(n_vis, ptr(u), ptr(v), ptr(w), ptr(vis), ptr(wt), n, fov, pa.numel(), ptr(pa),
                               ptr(pb), ptr(out), stream)


def test_dft_noalloc_matches_wst_dft_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06061_gb300 import build, wst

    build.build()
    lib = wst.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, fov = 1024, 0.2
    for seed, n_vis, n_pix in ((1, 30000, 4096), (2, 7000, 333)):
        u, v, w, vis, wt, pa, pb = _case(seed, n_vis, n_pix, n, fov)
        ref = torch.empty(n_pix, dtype=torch.complex64, device="cuda")
        wst.wst_dft(u, v, w, vis, n, fov, pa, pb, ref, weight=wt)
        got = torch.full((n_pix,), float("nan"), dtype=torch.complex64, device="cuda")
        assert _noalloc(lib, stream, n_vis, u, v, w, vis, wt, n, fov, pa, pb, got) == 0
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - r).max() <= TOL * np.abs(r).max()


def test_dft_noalloc_repeats_bit_for_bit_and_covers_edge_inputs():
    """The same inputs give the same bits (the blocks are summed in a fixed order); no
    weights equals unit weights; no visibilities gives zeros."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06061_gb300 import build, wst

    build.build()
    lib = wst.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, fov, n_vis, n_pix = 512, 0.15, 20000, 1000
    u, v, w, vis, wt, pa, pb = _case(4, n_vis, n_pix, n, fov)
    first = torch.full((n_pix,), float("nan"), dtype=torch.complex64, device="cuda")
    second = torch.full((n_pix,), float("nan"), dtype=torch.complex64, device="cuda")
    assert _noalloc(lib, stream, n_vis, u, v, w, vis, wt, n, fov, pa, pb, first) == 0
    assert _noalloc(lib, stream, n_vis, u, v, w, vis, wt, n, fov, pa, pb, second) == 0
    assert torch.equal(first.view(torch.float32), second.view(torch.float32))
    # weight = NULL: natural weights, against wst_dft with unit weights
    got = torch.full((n_pix,), float("nan"), dtype=torch.complex64, device="cuda")
    assert _noalloc(lib, stream, n_vis, u, v, w, vis, None, n, fov, pa, pb, got) == 0
    ref = torch.empty(n_pix, dtype=torch.complex64, device="cuda")
    wst.wst_dft(u, v, w, vis, n, fov, pa, pb, ref, weight=torch.ones_like(wt))
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    assert np.abs(g - r).max() <= TOL * np.abs(r).max()
    # n_vis = 0: the scratch still holds the last call's sums; the output must be zeros
    zero = torch.full((n_pix,), float("nan"), dtype=torch.complex64, device="cuda")
    assert _noalloc(lib, stream, 0, None, None, None, None, None, n, fov, pa, pb, zero) == 0
    assert torch.count_nonzero(zero).item() == 0


def test_dft_noalloc_rejects_too_many_pixels():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06061_gb300 import build, wst

    build.build()
    n_pix = wst.WST_DFT_NOALLOC_MAX_PIX + 1
    u, v, w, vis, wt, pa, pb = _case(3, 100, n_pix, 256, 0.1)
    out = torch.zeros(n_pix, dtype=torch.complex64, device="cuda")
    assert wst.wst_dft_noalloc(u, v, w, vis, 256, 0.1, pa, pb, out) == 5  # WST_ERR_UNSUPPORTED
    assert torch.count_nonzero(out).item() == 0
