"""The Kaiser-Bessel table helper against scipy's modified Bessel function (an
independent implementation) and the window's defining properties."""
import math

import numpy as np
import pytest

from paper_2301_06061_gb300 import kernels

special = pytest.importorskip("scipy.special")


def test_kaiser_bessel_table_matches_scipy_i0():
    W, beta, pc = 8, 12.25, 64
    t = kernels.kaiser_bessel_table(W, beta, pc)
    x = np.linspace(-W / 2, W / 2, W * pc + 1)
    ref = special.i0(beta * np.sqrt(np.clip(1 - (2 * x / W) ** 2, 0, None))) / special.i0(beta)
    assert t.dtype == np.float32 and t.size == W * pc + 1
    assert np.abs(t - ref).max() < 1e-7
    assert t[W * pc // 2] == 1.0 and np.array_equal(t, t[::-1])
    assert t[0] == pytest.approx(1.0 / special.i0(beta), rel=1e-6)  # the end points: I0(0) / I0(beta)


def test_kaiser_bessel_beta_formula():
    # Beatty et al. 2005, Eq. 5, by hand for W = 8: alpha = 2 -> pi sqrt(16 * 2.25 - 0.8)
    assert kernels.kaiser_bessel_beta(8, 2.0) == pytest.approx(math.pi * math.sqrt(35.2))
    assert kernels.kaiser_bessel_beta(8, 1.0) == pytest.approx(math.pi * math.sqrt(15.2))
    with pytest.raises(ValueError):
        kernels.kaiser_bessel_beta(1, 1.0)


# ------------------------------------------------------------------------------------------
# prolate spheroidal wave function (psi_0) table
# ------------------------------------------------------------------------------------------

def test_pswf_matches_scipy_prolate_angular_function():
    """psi_0(c, x) from the quadrature eigenproblem against scipy's prolate spheroidal
    angular function of the first kind (an independent series method), both scaled to
    1 at x = 0.  The series loses digits as c grows (its own eigen-relation residual is
    4e-8 at c = 6 pi, the quadrature's 1e-10), so the bound is 5e-8 of the peak, below
    the FP32 resolution of the tables."""
    for c in (kernels.pswf_c(8, 1.0), kernels.pswf_c(8, 2.0), kernels.pswf_c(6, 1.25)):
        x = np.linspace(-0.99, 0.99, 23)
        ref = np.array([special.pro_ang1(0, 0, c, v)[0] for v in x]) / special.pro_ang1(0, 0, c, 0.0)[0]
        assert np.abs(kernels.pswf_values(c, x) - ref).max() < 5e-8


def test_pswf_is_an_eigenfunction_of_the_finite_fourier_transform():
    """int_{-1}^{1} cos(c x t) psi(t) dt / psi(x) is the same number at every x (a finer,
    independent quadrature than the one that built psi)."""
    c = kernels.pswf_c(8, 1.5)
    t, w = np.polynomial.legendre.leggauss(300)
    psi_t = kernels.pswf_values(c, t)
    x = np.array([-0.95, -0.6, -0.25, 0.0, 0.3, 0.55, 0.9])
    ratio = (np.cos(c * np.outer(x, t)) @ (w * psi_t)) / kernels.pswf_values(c, x)
    assert ratio.std() < 1e-10 * abs(ratio.mean())


def _concentration(f, c):
    """Fraction of the energy of f's Fourier transform (f supported on [-1, 1]) in
    |omega| <= c, by quadrature in t and in omega and Parseval for the total."""
    t, wt = np.polynomial.legendre.leggauss(200)
    om, wo = np.polynomial.legendre.leggauss(200)
    om, wo = om * c, wo * c
    ft = np.exp(-1j * np.outer(om, t)) @ (wt * f(t))
    return float((wo * np.abs(ft) ** 2).sum() / (2 * np.pi * (wt * f(t) ** 2).sum()))


def test_pswf_has_the_most_concentrated_spectrum():
    """Slepian and Pollak: among functions on [-1, 1], psi_0 maximises the share of its
    spectrum in |omega| <= c.  It beats the Kaiser-Bessel window of the same shape
    parameter and the Gaussian, and every small perturbation of it lowers the share."""
    c = kernels.pswf_c(8, 1.0)
    psi = lambda t: kernels.pswf_values(c, t)
    best = _concentration(psi, c)
    kb = _concentration(lambda t: special.i0(c * np.sqrt(np.clip(1 - t * t, 0, None))), c)
    gauss = _concentration(lambda t: np.exp(-t * t / (2 * 0.22**2)), c)
    assert best > kb > 0.99 and best > gauss
    for h in (lambda t: t * t, lambda t: np.cos(3 * t), lambda t: 1 - t**4):
        assert _concentration(lambda t: psi(t) + 1e-3 * h(t), c) < best


def test_pswf_table_layout_and_band_parameter():
    W, pc = 8, 64
    c = kernels.pswf_c(W, 2.0)
    assert c == pytest.approx(math.pi * 8 * 0.75)  # pi W (1 - 1/(2 alpha)) by hand
    assert kernels.pswf_c(8, 1.0) == pytest.approx(4 * math.pi)
    with pytest.raises(ValueError):
        kernels.pswf_c(8, 0.5)
    t = kernels.pswf_table(W, c, pc)
    assert t.dtype == np.float32 and t.size == W * pc + 1
    assert t[W * pc // 2] == 1.0 and np.array_equal(t, t[::-1]) and np.all(t > 0)
    x = np.linspace(-W / 2, W / 2, W * pc + 1)
    assert np.abs(t - kernels.pswf_values(c, 2 * x / W)).max() < 1e-7
