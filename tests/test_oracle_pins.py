"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one oracle function to a closed form, a library routine the
oracle does not use, an exact identity, or brute force on tiny inputs, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from oracle import OracleConfig
from paper_2301_06061_gb300 import synth


def gauss_ft_closed(nu, sigma, W):
    """Fourier transform of the Gaussian truncated to [-W/2, W/2] (complex-erf closed form)."""
    nu = np.asarray(nu, dtype=np.float64)
    h = 0.5 * W
    c = 2j * np.pi * nu * sigma**2
    s2 = sigma * math.sqrt(2.0)
    val = special.erf((h - c) / s2) + special.erf((h + c) / s2)
    return sigma * math.sqrt(math.pi / 2.0) * np.exp(-2.0 * np.pi**2 * nu**2 * sigma**2) * val.real


def alias_ratio(nu, kernel_fn, ghat_fn, W, n_off=512):
    """Worst single-visibility aliasing error over sub-cell offsets g in [0, 1):

        eps(nu) = max_g | sum_{a<W} G(a - W/2 + g) e^{2 pi i (a - W/2 + g) nu} / Ghat(nu) - 1 |

    By Poisson summation the finite tap sum equals Ghat(nu) plus the aliased images
    Ghat(nu - k), k != 0, so this is the exact (u,v) aliasing ratio of one visibility.
    The maximum over 512 offsets is padded by 2% for the unsampled offsets.
    """
    nu = np.asarray(nu, dtype=np.float64)
    g = (np.arange(n_off) + 0.5) / n_off
    t = np.arange(W)[None, :] - W / 2 + g[:, None]  # (n_off, W) tap offsets
    gt = kernel_fn(t)
    ph = np.exp(2j * np.pi * t[None, :, :] * nu[:, None, None])  # (n_nu, n_off, W)
    s = (gt[None] * ph).sum(-1) / ghat_fn(nu)[:, None]
    return np.abs(s - 1).max(axis=1) * 1.02


def gauss_alias(nu, sigma, W):
    return alias_ratio(nu, lambda t: np.exp(-t**2 / (2 * sigma**2)),
                       lambda x: gauss_ft_closed(x, sigma, W), W)


# ------------------------------------------------------------------------------------------
# FFT (paper section 2: the per-plane transform of Eq. 2)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 4, 8, 16, 64, 256, 1024])
def test_fft1d_matches_pocketfft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    # positive exponent: numpy's unnormalised inverse transform
    np.testing.assert_allclose(oracle.fft1d(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-12 * n)
    np.testing.assert_allclose(oracle.fft1d(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * n)


def test_fft1d_textbook_dft():
    n = 32
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    mat = np.exp(2j * np.pi * np.outer(j, j) / n)
    np.testing.assert_allclose(oracle.fft1d(x, +1), mat @ x, atol=1e-12)


@pytest.mark.parametrize("sign", [+1, -1])
def test_fft2_centered_definition(sign):
    """F[b,a] = sum g[q,p] exp(sign 2 pi i ((p-N/2)(a-N/2) + (q-N/2)(b-N/2))/N)."""
    N = 16
    rng = np.random.default_rng(7)
    g = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    c = np.arange(N) - N // 2
    E = np.exp(sign * 2j * np.pi * np.outer(c, c) / N)  # E[a, p]
    expect = E @ g @ E.T  # rows: b via q, columns: a via p
    np.testing.assert_allclose(oracle.fft2_centered(g, sign), expect, atol=1e-11)


def test_fft2_centered_vs_numpy_shift():
    N = 64
    rng = np.random.default_rng(3)
    g = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    expect = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g))) * N * N
    np.testing.assert_allclose(oracle.fft2_centered(g, +1), expect, atol=1e-10)


# ------------------------------------------------------------------------------------------
# Kernel and its transform (Eq. 3; grid correction)
# ------------------------------------------------------------------------------------------

def test_gauss_legendre_exact_on_polynomials():
    for n in (4, 8, 16):
        x, w = oracle.gauss_legendre(n)
        for p in range(2 * n):
            exact = 0.0 if p % 2 else 2.0 / (p + 1)
            assert abs(np.sum(w * x**p) - exact) < 1e-14


@pytest.mark.parametrize("W,sigma", [(7, 0.875), (8, 0.925), (7, 1.3)])
def test_kernel_ft_gaussian_closed_form(W, sigma):
    cfg = OracleConfig(64, 0.1, 1, 0, 0, W, "gauss", sigma)
    nu = np.linspace(-0.5, 0.5, 41)
    np.testing.assert_allclose(oracle.kernel_ft(cfg, nu), gauss_ft_closed(nu, sigma, W),
                               rtol=1e-13, atol=1e-15)


def test_kernel_ft_es_against_adaptive_quadrature():
    W, beta = 8, 2.3 * 8
    cfg = OracleConfig(64, 0.1, 1, 0, 0, W, "es", beta)
    for nu in (0.0, 0.13, 0.31, 0.5):
        f = lambda x: math.exp(beta * (math.sqrt(max(0.0, 1 - (2 * x / W) ** 2)) - 1)) * math.cos(
            2 * math.pi * nu * x)
        ref, _ = integrate.quad(f, -W / 2, W / 2, epsabs=1e-14, epsrel=1e-13, limit=400)
        assert abs(oracle.kernel_ft(cfg, [nu])[0] - ref) < 1e-10 * max(1.0, abs(ref))


def test_kernel_ft_table_piecewise_linear_closed_form():
    W, L = 8, 8 * 16 + 1
    rng = np.random.default_rng(11)
    tab = rng.random(L)
    cfg = OracleConfig(64, 0.1, 1, 0, 0, W, "table", 0.0, tab)
    xs = np.linspace(-W / 2, W / 2, L)
    for nu in (0.0, 0.07, 0.25, 0.49):
        k = 2 * math.pi * nu
        tot = 0.0
        for i in range(L - 1):
            x0, x1 = xs[i], xs[i + 1]
            b = (tab[i + 1] - tab[i]) / (x1 - x0)
            a = tab[i] - b * x0
            if k == 0:
                tot += a * (x1 - x0) + b * (x1**2 - x0**2) / 2
            else:
                F = lambda x: a * math.sin(k * x) / k + b * (math.cos(k * x) / k**2 + x * math.sin(k * x) / k)
                tot += F(x1) - F(x0)
        assert abs(oracle.kernel_ft(cfg, [nu])[0] - tot) < 1e-12


def test_kernel_eval_table_interpolates():
    W, L = 8, 33
    tab = np.linspace(0, 1, L) ** 2
    cfg = OracleConfig(64, 0.1, 1, 0, 0, W, "table", 0.0, tab)
    xs = np.linspace(-W / 2, W / 2, L)
    for i in (0, 5, 31):
        mid = 0.5 * (xs[i] + xs[i + 1])
        assert abs(oracle.kernel_eval(cfg, mid) - 0.5 * (tab[i] + tab[i + 1])) < 1e-15
        assert abs(oracle.kernel_eval(cfg, xs[i]) - tab[i]) < 1e-15


# ------------------------------------------------------------------------------------------
# Phase screen term n - 1 (Eq. 1-2)
# ------------------------------------------------------------------------------------------

def test_n_minus_one_high_precision():
    getcontext().prec = 60
    for l, m in [(0.0, 0.0), (1e-4, -2e-4), (0.05, 0.05), (0.25, -0.25), (0.6, 0.7)]:
        r2 = Decimal(l) ** 2 + Decimal(m) ** 2
        exact = float((Decimal(1) - r2).sqrt() - Decimal(1))
        got = oracle.n_minus_one(l, m)
        assert abs(got - exact) <= 2e-16 * max(abs(exact), 1e-300) + 1e-300
    assert math.isnan(oracle.n_minus_one(0.8, 0.7))


# ------------------------------------------------------------------------------------------
# Placement: nearest w-plane and kernel footprint (Eq. 3 discretisation)
# ------------------------------------------------------------------------------------------

def test_locate_exact_rules():
    N, fov, W, n_w = 256, 0.1, 7, 8
    rng = np.random.default_rng(5)
    n = 4000
    u = rng.uniform(-1400, 1400, n).astype(np.float32)
    v = rng.uniform(-1400, 1400, n).astype(np.float32)
    w = rng.uniform(-220, 220, n).astype(np.float32)
    vis = np.ones(n, np.complex64)
    u[:3] = [np.nan, 0, 0]
    w[3] = np.inf
    vis[4] = np.nan
    cfg = OracleConfig(N, fov, n_w, -200.0, 200.0, W)
    k, i0, j0, st = oracle.locate(cfg, u, v, w, vis)
    assert st[0] == 2 and st[3] == 2 and st[4] == 2
    F = Fraction
    dw = (F(200) - F(-200)) / n_w
    for j in range(5, n):
        x = F(N, 2) + F(float(u[j])) * F(fov)
        y = F(N, 2) + F(float(v[j])) * F(fov)
        ci = math.ceil(x - F(W, 2))
        cj = math.ceil(y - F(W, 2))
        inside = ci >= 0 and cj >= 0 and ci + W <= N and cj + W <= N
        if not inside:
            assert st[j] == 1, j
            continue
        assert st[j] == 0
        assert int(i0[j]) == ci and int(j0[j]) == cj
        # every tap offset lies in [-W/2, W/2)
        assert x - F(W, 2) <= int(i0[j]) < x - F(W, 2) + 1
        kk = math.floor((F(float(w[j])) - F(-200)) / dw)
        kk = min(max(kk, 0), n_w - 1)
        assert int(k[j]) == kk


def _plane_boundary_cases(w_min, w_max, n_w):
    """FP32 w on, and 1 or 2 FP32 steps either side of, every interior plane boundary
    w_min + k (w_max - w_min) / n_w (the FP32 values nearest to each boundary)."""
    F = Fraction
    ws = []
    for k in range(1, n_w):
        b = F(w_min) + k * (F(w_max) - F(w_min)) / n_w
        c = np.float32(float(b))
        ws += [c, np.nextafter(c, np.float32(np.inf)), np.nextafter(c, np.float32(-np.inf))]
        ws += [np.nextafter(ws[-2], np.float32(np.inf)), np.nextafter(ws[-1], np.float32(-np.inf))]
    return np.array(ws, np.float32)


@pytest.mark.parametrize("w_min,w_max,n_w,n_down", [
    (-256.0, 256.0, 32, 0),         # dyadic N_w / range: the product is exact
    (-200.0, 200.0, 8, 0),          # the tiny workload's planes; N_w / range rounds up in FP64
    (-6547.25, 6728.5, 32, 0),      # a range like the benchmark's: dw dyadic, N_w / range rounds down
    (-1000.0, 2000.0, 3, 0),        # dw = 1000: boundaries exact in FP32, N_w / range rounds up
    (-0.75, 6.0, 27, 0),            # N_w / range = 4: dyadic again
    (-3.3333332538604736, 6.6666669845581055, 48, 1),  # FP32 end points; rounds down, one hit goes down
])
def test_locate_plane_rule_at_exact_boundaries(w_min, w_max, n_w, n_down):
    """The plane rule k = floor(fl(fl(w - w_min) * fl(N_w / (w_max - w_min)))) (closest
    plane, section 2; FP64, one product per visibility) against exact rational arithmetic
    q = (w - w_min) N_w / (w_max - w_min), k_exact = floor(q), with w on, and 1-2 FP32
    steps from, each boundary.  Three FP64 roundings (difference, scale, product) move
    q by at most 2^-50 |q|, so:
      * where q is farther than that from an integer, the exact plane is taken;
      * where q is within that of an integer m but not equal to it (here: the boundary at
        w = 0, whose FP32 neighbours are subnormal, so fl(w - w_min) = -w_min), the
        visibility goes to m - 1 or m -- both planes are closest to within FP64 rounding;
      * where q is exactly an integer m (w exactly on a boundary), the visibility goes to
        the upper plane m when fl(N_w / range) >= N_w / range (a dyadic or rounded-up
        scale), and may go to m - 1 only when the scale rounded down.
    The GPU sort takes the same decision as this rule, bit for bit."""
    F = Fraction
    w = _plane_boundary_cases(w_min, w_max, n_w)
    cfg = OracleConfig(64, 0.1, n_w, w_min, w_max, 7)
    z = np.zeros(w.size, np.float32)
    k, _, _, st = oracle.locate(cfg, z, z, w, np.ones(w.size, np.complex64))
    assert np.all(st == 0)
    scale_exact = F(n_w) / (F(w_max) - F(w_min))
    scale_rounded_down = F(n_w / (w_max - w_min)) < scale_exact
    hits = near = down = 0
    for j in range(w.size):
        q = (F(float(w[j])) - F(w_min)) * scale_exact
        m = round(q)
        got = int(k[j])
        if q == m:  # exactly on a boundary
            hits += 1
            if scale_rounded_down:
                assert got in (m - 1, m), (w[j], got, m)
                down += got == m - 1
            else:
                assert got == min(m, n_w - 1), (w[j], got, m)
        elif abs(q - m) <= F(1, 2**50) * max(abs(q), 1):
            near += 1
            assert got in (m - 1, m), (w[j], got, m)
        else:
            assert got == min(max(math.floor(q), 0), n_w - 1), (w[j], got, q)
    # the dyadic configurations and the exact-dw one really put w on the boundaries
    if (w_min, n_w) in ((-256.0, 32), (-1000.0, 3), (-0.75, 27)):
        assert hits == n_w - 1
    # a boundary at w = 0 has subnormal neighbours: four cases within FP64 rounding
    if (w_min, n_w) in ((-256.0, 32), (-200.0, 8), (-1000.0, 3), (-0.75, 27)):
        assert near == 4
    # exact hits that the rounded-down scale sends to the lower plane (w = -0.2083331794
    # on the boundary of planes 14 and 15 of the last configuration)
    assert down == n_down


def test_plane_centres_cell_centred():
    cfg = OracleConfig(64, 0.1, 8, -200.0, 200.0, 7)
    assert [oracle.plane_centre(cfg, k) for k in range(8)] == [-175, -125, -75, -25, 25, 75, 125, 175]


# ------------------------------------------------------------------------------------------
# Gridding (Eq. 3)
# ------------------------------------------------------------------------------------------

def test_grid_cell_centre_visibility_is_separable_gaussian():
    N, fov, W, sigma = 64, 0.1, 7, 0.875
    cfg = OracleConfig(N, fov, 1, -1.0, 1.0, W, "gauss", sigma)
    # u chosen so that x = N/2 + u*fov = 40 exactly (u = 80 wavelengths)
    u = np.array([80.0], np.float32)
    v = np.array([-50.0], np.float32)  # y = 27
    w = np.array([0.0], np.float32)
    vis = np.array([2.0 - 1.0j], np.complex64)
    g = oracle.grid(cfg, u, v, w, vis)[0]
    off = np.arange(-3, 4)
    prof = np.exp(-off**2 / (2 * sigma**2))
    expect = np.zeros((N, N), complex)
    expect[27 - 3:27 + 4, 40 - 3:40 + 4] = (2 - 1j) * np.outer(prof, prof)
    np.testing.assert_allclose(g, expect, atol=1e-15)


def test_grid_weights_and_plane_routing():
    N, fov = 64, 0.1
    cfg = OracleConfig(N, fov, 4, -100.0, 100.0, 7)
    u = np.array([10.0, 10.0], np.float32)
    v = np.array([5.0, 5.0], np.float32)
    w = np.array([-99.0, 60.0], np.float32)  # planes 0 and 3
    vis = np.array([1 + 1j, 3.0], np.complex64)
    wt = np.array([0.5, 2.0], np.float32)
    g = oracle.grid(cfg, u, v, w, vis, wt)
    g1 = oracle.grid(cfg, u[:1], v[:1], w[:1], np.array([1.0], np.complex64))
    np.testing.assert_allclose(g[0], 0.5 * (1 + 1j) * g1[0], atol=1e-15)
    np.testing.assert_allclose(g[3], 6.0 * g1[0], atol=1e-15)
    assert np.all(g[1] == 0) and np.all(g[2] == 0)


# ------------------------------------------------------------------------------------------
# The image: brute-force DFT, flat image, linearity, Hermitian symmetry (Eq. 1-3)
# ------------------------------------------------------------------------------------------

def test_predict_and_dft_point_source_peak():
    """A unit point source at a pixel centre: the direct transform there equals n_vis."""
    N, fov = 64, 0.1
    rng = np.random.default_rng(2)
    u, v, w = synth.disk_uvw(500, 0.45 * N / fov, 150.0, rng)
    a, b = 40, 21
    l, m = (a - N // 2) * fov / N, (b - N // 2) * fov / N
    V = oracle.predict_points(u, v, w, [l], [m], [1.0]).astype(np.complex64)
    d = oracle.dft_pixels(u, v, w, V, N, fov, [a], [b])
    assert abs(d[0] - 500) < 1e-3  # complex64 rounding of V
    # sign: Eq. 1 carries exp(-2 pi i ...), the image exp(+2 pi i ...)
    Vd = oracle.predict_points(u, v, w, [l], [m], [1.0])
    assert np.isclose(Vd[0], np.exp(-2j * np.pi * (u[0] * l + v[0] * m + w[0] * oracle.n_minus_one(l, m))))


def _snapped_case(N=64, fov=0.1, n_w=5, n_vis=300, W=7, sigma=0.875, seed=9):
    rng = np.random.default_rng(seed)
    u, v, w = synth.disk_uvw(n_vis, 0.45 * N / fov, 200.0, rng)
    cfg = OracleConfig(N, fov, n_w, -200.0, 200.0, W, "gauss", sigma)
    k, _, _, st = oracle.locate(cfg, u, v, w, np.ones(n_vis, np.complex64))
    wk = np.array([oracle.plane_centre(cfg, int(kk)) for kk in k])
    w = np.where(st == 0, wk, w).astype(np.float32)  # centres of [-200,200]/5 are exact
    vis = synth.random_visibilities(n_vis, rng)
    return cfg, u, v, w, vis


def test_image_vs_dft_within_aliasing_bound():
    """w snapped to plane centres: the only error left is (u,v) aliasing, bounded by
    sum_j |V_j| (e_a + e_b + e_a e_b), e(nu) = sum_{k!=0} |Ghat(nu+k)|/|Ghat(nu)|."""
    cfg, u, v, w, vis = _snapped_case()
    N = cfg.n
    img = oracle.image(cfg, u, v, w, vis)
    a, b = np.meshgrid(np.arange(N), np.arange(N))
    d = oracle.dft_pixels(u, v, w, vis, N, cfg.fov, a.ravel(), b.ravel()).reshape(N, N)
    nu = (np.arange(N) - N // 2) / N
    e = gauss_alias(nu, cfg.kparam, cfg.support)
    bound = np.abs(vis).astype(np.float64).sum() * (e[None, :] + e[:, None] + e[None, :] * e[:, None])
    err = np.abs(img - d)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-9)
    # the bound is tight enough to mean something in the central half
    c = slice(N // 4, 3 * N // 4)
    assert err[c, c].max() < 2e-3 * np.abs(d).max()


def test_image_unsnapped_w_error_bound():
    """With w not snapped, add |V_j| 2 pi |w_j - w_k| |t| per visibility."""
    N, fov, n_w = 64, 0.1, 4
    rng = np.random.default_rng(4)
    u, v, w = synth.disk_uvw(300, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(300, rng)
    cfg = OracleConfig(N, fov, n_w, -200.0, 200.0, 7)
    img = oracle.image(cfg, u, v, w, vis)
    k, _, _, st = oracle.locate(cfg, u, v, w, vis)
    dwk = np.abs(w - np.array([oracle.plane_centre(cfg, int(x)) for x in k]))
    pix = np.arange(N)
    a, b = np.meshgrid(pix, pix)
    d = oracle.dft_pixels(u, v, w, vis, N, fov, a.ravel(), b.ravel()).reshape(N, N)
    dl = fov / N
    t = np.vectorize(oracle.n_minus_one)((a - N // 2) * dl, (b - N // 2) * dl)
    nu = (pix - N // 2) / N
    e = gauss_alias(nu, cfg.kparam, cfg.support)
    ea = e[None, :] + e[:, None] + e[None, :] * e[:, None]
    av = np.abs(vis).astype(np.float64)
    bound = av.sum() * ea + (1 + ea) * np.abs(t) * 2 * np.pi * (av * dwk).sum()
    assert np.all(np.abs(img - d) <= bound * (1 + 1e-9) + 1e-9)


def test_single_visibility_flat_image():
    """One visibility V = 1 at (0,0,0) on the centre plane: D = 1 up to the aliasing ratio,
    and exactly g(nu_a) g(nu_b) / (Ghat(nu_a) Ghat(nu_b)) with g the sampled-kernel series."""
    N, fov, W, sigma = 64, 0.1, 7, 0.875
    cfg = OracleConfig(N, fov, 3, -30.0, 30.0, W, "gauss", sigma)
    img = oracle.image(cfg, [0.0], [0.0], [0.0], np.array([1.0], np.complex64))
    nu = (np.arange(N) - N // 2) / N
    s = np.arange(-3, 4)
    gser = (np.exp(-s**2 / (2 * sigma**2))[None, :] * np.exp(2j * np.pi * np.outer(nu, s))).sum(1)
    gh = gauss_ft_closed(nu, sigma, W)
    np.testing.assert_allclose(img, np.outer(gser / gh, gser / gh), atol=1e-12)
    e = gauss_alias(nu, sigma, W)
    assert np.all(np.abs(img - 1) <= (e[None, :] + e[:, None] + np.outer(e, e)) * (1 + 1e-9))
    c = slice(N // 4, 3 * N // 4)
    assert np.abs(img[c, c] - 1).max() < 3e-3


def test_point_source_peak_at_pixel():
    N, fov = 64, 0.1
    rng = np.random.default_rng(8)
    u, v, w = synth.disk_uvw(2000, 0.45 * N / fov, 0.0, rng)
    w[:] = 0.0
    a, b = 37, 25
    l, m = (a - N // 2) * fov / N, (b - N // 2) * fov / N
    V = oracle.predict_points(u, v, w, [l], [m], [1.0]).astype(np.complex64)
    cfg = OracleConfig(N, fov, 1, -1.0, 1.0, 7)
    img = oracle.image(cfg, u, v, w, V)
    assert np.unravel_index(np.argmax(img.real), img.shape) == (b, a)


def test_image_linearity():
    N, fov = 64, 0.1
    rng = np.random.default_rng(12)
    u, v, w = synth.disk_uvw(400, 0.45 * N / fov, 200.0, rng)
    v1 = synth.random_visibilities(400, rng)
    v2 = synth.random_visibilities(400, rng)
    cfg = OracleConfig(N, fov, 4, -200.0, 200.0, 7)
    al, be = 0.7 - 0.2j, -1.3 + 0.5j
    comb = (al * v1.astype(complex) + be * v2.astype(complex))
    # complex64 rounding of the combination is the only difference
    lhs = oracle.image(cfg, u, v, w, comb.astype(np.complex64))
    rhs = al * oracle.image(cfg, u, v, w, v1) + be * oracle.image(cfg, u, v, w, v2)
    ref = oracle.image(cfg, u, v, w, comb.astype(np.complex64))
    np.testing.assert_allclose(lhs, ref, atol=0)
    assert np.abs(lhs - rhs).max() < 1e-6 * np.abs(rhs).max()


def test_image_hermitian_symmetry():
    N, fov = 64, 0.1
    rng = np.random.default_rng(13)
    # radius 0.4 N/FoV: the footprint and its mirror both stay on the grid
    u, v, w = synth.disk_uvw(300, 0.4 * N / fov, 180.0, rng)
    vis = synth.random_visibilities(300, rng)
    U = np.concatenate([u, -u])
    Vv = np.concatenate([v, -v])
    Wv = np.concatenate([w, -w])
    VV = np.concatenate([vis, np.conj(vis)])
    cfg = OracleConfig(N, fov, 6, -200.0, 200.0, 7)
    k, _, _, st = oracle.locate(cfg, U, Vv, Wv, VV)
    assert np.all(st == 0) and np.all(k[:300] + k[300:] == 5)
    img = oracle.image(cfg, U, Vv, Wv, VV)
    assert np.abs(img.imag).max() < 1e-10 * np.abs(img.real).max()


def test_image_pixels_matches_planes():
    N, fov = 64, 0.1
    rng = np.random.default_rng(14)
    u, v, w = synth.disk_uvw(300, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(300, rng)
    wt = rng.uniform(0.5, 2.0, 300).astype(np.float32)
    cfg = OracleConfig(N, fov, 4, -200.0, 200.0, 8, "gauss", 0.925)
    img = oracle.image(cfg, u, v, w, vis, wt)
    pa = rng.integers(0, N, 50)
    pb = rng.integers(0, N, 50)
    pix = oracle.image_pixels(cfg, u, v, w, vis, pa, pb, wt)
    np.testing.assert_allclose(pix, img[pb, pa], atol=1e-10 * np.abs(img).max())


def test_outside_unit_sphere_is_zero():
    N, fov = 64, 2.4  # corners have l^2 + m^2 > 1
    cfg = OracleConfig(N, fov, 1, -1.0, 1.0, 7)
    img = oracle.image(cfg, [0.0], [0.0], [0.0], np.array([1.0], np.complex64))
    dl = fov / N
    a, b = np.meshgrid(np.arange(N), np.arange(N))
    r2 = ((a - N // 2) * dl) ** 2 + ((b - N // 2) * dl) ** 2
    assert np.all(img[r2 >= 1] == 0) and np.all(img[r2 < 1] != 0)


# ------------------------------------------------------------------------------------------
# Adjoint and kernel gradient
# ------------------------------------------------------------------------------------------

def test_degrid_is_adjoint_dot_product():
    N, fov = 64, 0.1
    rng = np.random.default_rng(21)
    u, v, w = synth.disk_uvw(200, 0.45 * N / fov, 200.0, rng)
    wt = rng.uniform(0.5, 2.0, 200).astype(np.float32)
    x = synth.random_visibilities(200, rng)
    cfg = OracleConfig(N, fov, 4, -200.0, 200.0, 7)
    y = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    for corr in (True, False):
        Ax = oracle.image(cfg, u, v, w, x, wt, correct=corr)
        Ahy = oracle.degrid(cfg, u, v, w, x, y, wt, correct=corr)
        lhs = np.vdot(y, Ax)  # <y, A x>
        rhs = np.vdot(Ahy, x.astype(complex))  # <A^H y, x>
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_kernel_grad_finite_differences():
    N, fov, W = 64, 0.1, 8
    L = W * 4 + 1
    rng = np.random.default_rng(22)
    u, v, w = synth.disk_uvw(60, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(60, rng)
    tab = np.exp(-np.linspace(-W / 2, W / 2, L) ** 2 / (2 * 0.925**2))
    cfg = OracleConfig(N, fov, 3, -200.0, 200.0, W, "table", 0.0, tab)
    dU = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    g = oracle.kernel_grad(cfg, u, v, w, vis, dU)

    def loss(t):
        c = OracleConfig(N, fov, 3, -200.0, 200.0, W, "table", 0.0, t)
        return np.real(np.vdot(dU, oracle.image(c, u, v, w, vis, correct=False)))

    h = 1e-3
    for i in (0, 3, L // 2, L - 2, L - 1):
        tp, tm = tab.copy(), tab.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)  # exact for a loss quadratic in the table
        assert abs(fd - g[i]) < 1e-8 * max(1.0, np.abs(g).max())


# ------------------------------------------------------------------------------------------
# the w-folding variant (not in the paper): Hermitian mirror of the w < 0 visibilities
# ------------------------------------------------------------------------------------------

def test_fold_keeps_the_real_part_of_the_direct_transform():
    """A mirrored visibility (-u, -v, -w, conj V) adds the complex conjugate of the original
    term, so Re of the exact dirty image is unchanged and Im is not."""
    N, fov = 64, 0.1
    rng = np.random.default_rng(21)
    u, v, w = synth.disk_uvw(400, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(400, rng)
    fu, fv, fw, fvis = oracle.fold_w(u, v, w, vis)
    assert np.all(fw >= 0) and np.array_equal(np.abs(fw), np.abs(w)) and np.array_equal(fu == u, w >= 0)
    pix = np.arange(N)
    a, b = np.meshgrid(pix, pix)
    d = oracle.dft_pixels(u, v, w, vis, N, fov, a.ravel(), b.ravel())
    df = oracle.dft_pixels(fu, fv, fw, fvis, N, fov, a.ravel(), b.ravel())
    scale = np.abs(d).max()
    assert np.abs(df.real - d.real).max() <= 1e-12 * scale
    assert np.abs(df.imag - d.imag).max() > 1e-3 * scale


def test_fold_image_within_half_range_w_bound():
    """The folded w-stacking image approximates Re of the direct transform within the same
    per-visibility bound as the unfolded one, with the plane offsets of the folded range
    (half the plane spacing at the same number of planes)."""
    N, fov, n_w = 64, 0.1, 4
    rng = np.random.default_rng(22)
    u, v, w = synth.disk_uvw(300, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(300, rng)
    fu, fv, fw, fvis = oracle.fold_w(u, v, w, vis)
    lo, hi = oracle.resolve_w_range(fw, 0.0, 0.0)
    assert lo >= 0 and hi == float(np.abs(w).max())
    cfg = OracleConfig(N, fov, n_w, lo, hi, 7)
    img = oracle.image(cfg, fu, fv, fw, fvis)
    k, _, _, st = oracle.locate(cfg, fu, fv, fw, fvis)
    assert np.all(st == 0)
    dwk = np.abs(fw - np.array([oracle.plane_centre(cfg, int(x)) for x in k]))
    assert dwk.max() <= (hi - lo) / n_w / 2 * (1 + 1e-12)
    pix = np.arange(N)
    a, b = np.meshgrid(pix, pix)
    d = oracle.dft_pixels(u, v, w, vis, N, fov, a.ravel(), b.ravel()).reshape(N, N)
    dl = fov / N
    t = np.vectorize(oracle.n_minus_one)((a - N // 2) * dl, (b - N // 2) * dl)
    e = gauss_alias((pix - N // 2) / N, cfg.kparam, cfg.support)
    ea = e[None, :] + e[:, None] + e[None, :] * e[:, None]
    av = np.abs(vis).astype(np.float64)
    bound = av.sum() * ea + (1 + ea) * np.abs(t) * 2 * np.pi * (av * dwk).sum()
    assert np.all(np.abs(img.real - d.real) <= bound * (1 + 1e-9) + 1e-9)


# ------------------------------------------------------------------------------------------
# the oversampled-grid variant (not in the paper): a 2N grid, the central N x N kept
# ------------------------------------------------------------------------------------------

def test_oversampled_image_within_half_band_aliasing_bound():
    """w snapped to plane centres: the oversampled image's pixels are the grid's central
    half, |nu| <= 1/4 on the 2N grid, so the aliasing bound sum|V| (e_a + e_b + e_a e_b)
    with e taken there holds over the WHOLE image, and is small everywhere -- where the
    plain grid's edge pixels alias by design."""
    cfg, u, v, w, vis = _snapped_case()
    N = cfg.n
    img = oracle.image_oversampled(cfg, 2, u, v, w, vis)
    a, b = np.meshgrid(np.arange(N), np.arange(N))
    d = oracle.dft_pixels(u, v, w, vis, N, cfg.fov, a.ravel(), b.ravel()).reshape(N, N)
    nu = (np.arange(N) + N // 2 - N) / (2 * N)  # grid index a + N/2 on the 2N grid
    assert np.abs(nu).max() <= 0.25
    e = gauss_alias(nu, cfg.kparam, cfg.support)
    bound = np.abs(vis).astype(np.float64).sum() * (e[None, :] + e[:, None] + e[None, :] * e[:, None])
    err = np.abs(img - d)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-9)
    plain = np.abs(oracle.image(cfg, u, v, w, vis) - d)
    assert err.max() < 2e-3 * np.abs(d).max() and err.max() * 20 < plain.max()


def test_oversampled_degrid_is_adjoint_dot_product():
    """<y, A_os x> = <A_os^H y, x> for the oversampled image (crop of the 2N-grid image)
    and its adjoint (zero-pad, then the 2N-grid degridding), with and without the grid
    correction."""
    N, fov = 32, 0.1
    rng = np.random.default_rng(23)
    u, v, w = synth.disk_uvw(150, 0.45 * N / fov, 200.0, rng)
    wt = rng.uniform(0.5, 2.0, 150).astype(np.float32)
    x = synth.random_visibilities(150, rng)
    cfg = OracleConfig(N, fov, 3, -200.0, 200.0, 7)
    y = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    for corr in (True, False):
        Ax = oracle.image_oversampled(cfg, 2, u, v, w, x, wt, correct=corr)
        Ahy = oracle.degrid_oversampled(cfg, 2, u, v, w, x, y, wt, correct=corr)
        lhs = np.vdot(y, Ax)
        rhs = np.vdot(Ahy, x.astype(complex))
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # a zero image has a zero adjoint (nothing outside the N x N image enters)
    assert np.all(oracle.degrid_oversampled(cfg, 2, u, v, w, x, np.zeros((N, N)), wt) == 0)


def test_oversampled_kernel_grad_finite_differences():
    N, fov, W = 32, 0.1, 8
    L = W * 4 + 1
    rng = np.random.default_rng(24)
    u, v, w = synth.disk_uvw(50, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(50, rng)
    tab = np.exp(-np.linspace(-W / 2, W / 2, L) ** 2 / (2 * 0.925**2))
    cfg = OracleConfig(N, fov, 3, -200.0, 200.0, W, "table", 0.0, tab)
    dU = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    g = oracle.kernel_grad_oversampled(cfg, 2, u, v, w, vis, dU)

    def loss(t):
        c = OracleConfig(N, fov, 3, -200.0, 200.0, W, "table", 0.0, t)
        return np.real(np.vdot(dU, oracle.image_oversampled(c, 2, u, v, w, vis, correct=False)))

    h = 1e-3
    for i in (0, 5, L // 2, L - 3, L - 1):
        tp, tm = tab.copy(), tab.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)  # exact for a loss quadratic in the table
        assert abs(fd - g[i]) < 1e-8 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("N,M", [(100, 128), (170, 256), (204, 256)])
def test_image_on_a_grid_of_any_oversampling_within_aliasing_bound(N, M):
    """Oversampling factor M/N between 1 and 2 (1.28, 1.51, 1.25), N not a power of two:
    image pixel a is grid pixel a + (M - N)/2, at frequency nu = (a - N/2)/M, |nu| <=
    N/(2M); with w snapped, the direct transform lies within sum|V| (e_a + e_b + e_a e_b)
    of the image over the WHOLE image, e taken at those frequencies."""
    fov, n_vis = 0.1, 300
    rng = np.random.default_rng(9)
    u, v, w = synth.disk_uvw(n_vis, 0.45 * N / fov, 200.0, rng)
    cfg = OracleConfig(N, fov, 5, -200.0, 200.0, 7, "gauss", 0.875)
    k, _, _, st = oracle.locate(cfg, u, v, w, np.ones(n_vis, np.complex64))
    assert np.all(st == 0)
    w = np.array([oracle.plane_centre(cfg, int(kk)) for kk in k], np.float32)
    vis = synth.random_visibilities(n_vis, rng)
    img = oracle.image_on_grid(cfg, M, u, v, w, vis)
    assert img.shape == (N, N)
    a, b = np.meshgrid(np.arange(N), np.arange(N))
    d = oracle.dft_pixels(u, v, w, vis, N, fov, a.ravel(), b.ravel()).reshape(N, N)
    nu = (np.arange(N) - N // 2) / M
    e = gauss_alias(nu, cfg.kparam, cfg.support)
    bound = np.abs(vis).astype(np.float64).sum() * (e[None, :] + e[:, None] + e[None, :] * e[:, None])
    assert np.all(np.abs(img - d) <= bound * (1 + 1e-9) + 1e-9)
    # a wider grid for the same image keeps lower frequencies only: a smaller error
    wide = oracle.image_on_grid(cfg, 4 * M, u, v, w, vis)
    assert np.abs(wide - d).max() * 5 < np.abs(img - d).max()


def test_grid_config_is_the_plain_config_scaled_and_checks_its_inputs():
    cfg = OracleConfig(100, 0.1, 3, -1.0, 1.0)
    g = oracle.grid_config(cfg, 128)
    assert g.n == 128 and g.fov == 0.1 * 128 / 100 and g.n_w == 3
    assert oracle.grid_config(OracleConfig(64, 0.1, 3, -1.0, 1.0), 128).fov == 0.2  # exact
    with pytest.raises(ValueError):
        oracle.grid_config(cfg, 96)  # not a power of two
    with pytest.raises(ValueError):
        oracle.grid_config(cfg, 64)  # smaller than the image
    u = v = w = np.zeros(1, np.float32)
    with pytest.raises(ValueError):
        oracle.image_on_grid(OracleConfig(101, 0.1, 1, -1.0, 1.0), 128, u, v, w, np.ones(1, np.complex64))


def test_degrid_on_grid_is_adjoint_dot_product():
    """<y, A x> = <A^H y, x> for the image cropped from a grid of 1.28 N cells (N = 50)."""
    N, M, fov = 50, 64, 0.1
    rng = np.random.default_rng(25)
    u, v, w = synth.disk_uvw(150, 0.45 * N / fov, 200.0, rng)
    wt = rng.uniform(0.5, 2.0, 150).astype(np.float32)
    x = synth.random_visibilities(150, rng)
    cfg = OracleConfig(N, fov, 3, -200.0, 200.0, 7)
    y = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    for corr in (True, False):
        Ax = oracle.image_on_grid(cfg, M, u, v, w, x, wt, correct=corr)
        Ahy = oracle.degrid_on_grid(cfg, M, u, v, w, x, y, wt, correct=corr)
        assert abs(np.vdot(y, Ax) - np.vdot(Ahy, x.astype(complex))) < 1e-11 * abs(np.vdot(y, Ax))


def test_kernel_grad_on_grid_finite_differences():
    N, M, fov, W = 50, 64, 0.1, 8
    L = W * 4 + 1
    rng = np.random.default_rng(26)
    u, v, w = synth.disk_uvw(50, 0.45 * N / fov, 200.0, rng)
    vis = synth.random_visibilities(50, rng)
    tab = np.exp(-np.linspace(-W / 2, W / 2, L) ** 2 / (2 * 0.925**2))
    cfg = OracleConfig(N, fov, 3, -200.0, 200.0, W, "table", 0.0, tab)
    dU = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    g = oracle.kernel_grad_on_grid(cfg, M, u, v, w, vis, dU)

    def loss(t):
        c = OracleConfig(N, fov, 3, -200.0, 200.0, W, "table", 0.0, t)
        return np.real(np.vdot(dU, oracle.image_on_grid(c, M, u, v, w, vis, correct=False)))

    h = 1e-3
    for i in (0, 5, L // 2, L - 3, L - 1):
        tp, tm = tab.copy(), tab.copy()
        tp[i] += h
        tm[i] -= h
        assert abs((loss(tp) - loss(tm)) / (2 * h) - g[i]) < 1e-8 * max(1.0, np.abs(g).max())


# ------------------------------------------------------------------------------------------
# inputs by row and channel (the layout of the LOFAR datasets of section 4)
# ------------------------------------------------------------------------------------------

def test_expand_rows_exact_products_and_order():
    """Products of dyadic numbers are exact, so every coordinate is known by hand; the
    channel index runs fastest and the last row may be partial."""
    rows = np.array([[3.0, -5.0, 0.25], [-7.0, 1.5, -2.0]])
    scale = np.array([0.5, 2.0, 1.25])
    u, v, w = oracle.expand_rows(rows, scale, 5)
    np.testing.assert_array_equal(u, np.float32([1.5, 6.0, 3.75, -3.5, -14.0]))
    np.testing.assert_array_equal(v, np.float32([-2.5, -10.0, -6.25, 0.75, 3.0]))
    np.testing.assert_array_equal(w, np.float32([0.125, 0.5, 0.3125, -1.0, -4.0]))
    assert all(a.dtype == np.float32 for a in (u, v, w))
    with pytest.raises(ValueError):
        oracle.expand_rows(rows, scale, 7)


def test_expand_rows_rounds_the_fp64_product_once():
    """(1 + 2^-24 + 2^-30)(1 - 2^-30) = 1 + 2^-24 - 2^-54 - 2^-60: FP64 rounds it to
    1 + 2^-24, which FP32 rounds (tie to even) to 1.  Rounding the factors to FP32
    first gives (1 + 2^-23) * 1 instead."""
    x = 1.0 + 2.0 ** -24 + 2.0 ** -30
    s = 1.0 - 2.0 ** -30
    exact = Fraction(x) * Fraction(s)
    assert exact == 1 + Fraction(1, 2 ** 24) - Fraction(1, 2 ** 54) - Fraction(1, 2 ** 60)
    u, v, w = oracle.expand_rows([[x, -x, x]], [s], 1)
    assert u[0] == np.float32(1.0) and v[0] == np.float32(-1.0) and w[0] == np.float32(1.0)
    assert np.float32(x) * np.float32(s) == np.float32(1.0 + 2.0 ** -23)


def test_expand_rows_matches_the_workload_tracks():
    """The track generator's per-visibility coordinates and its rows x channels agree
    (the bench passes the same workload either way)."""
    work = synth.array(n_dumps=6)
    u, v, w = oracle.expand_rows(work.rows_m, work.chan_scale, work.n_vis)
    np.testing.assert_array_equal(u, work.u)
    np.testing.assert_array_equal(v, work.v)
    np.testing.assert_array_equal(w, work.w)
    assert work.n_vis == work.rows_m.shape[0] * work.chan_scale.size
