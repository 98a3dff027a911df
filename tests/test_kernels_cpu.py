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
