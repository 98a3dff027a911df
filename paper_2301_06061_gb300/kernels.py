"""Tabulated convolution kernels for WST_KERNEL_TABLE (section 2, Eq. 3: the kernel is the
imager's free choice; the paper uses a Gaussian of 7 cells and names better kernels as
future work in its conclusions).

``kaiser_bessel_table``: the Kaiser-Bessel window G(x) = I0(beta sqrt(1 - (2x/W)^2)) /
I0(beta) on |x| <= W/2, sampled at ``per_cell`` points per cell (piecewise-linear between
samples, as the library interpolates every table).  ``kaiser_bessel_beta`` is the
shape parameter of Beatty, Nishimura & Pauly (IEEE TMI 24, 2005, Eq. 5) for a grid
oversampled by ``alpha``: beta = pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8).
Host-side table construction only; the gridding runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np


def kaiser_bessel_beta(support: int, alpha: float = 1.0) -> float:
    x = (support / alpha) ** 2 * (alpha - 0.5) ** 2 - 0.8
    if x <= 0:
        raise ValueError("support too small for this oversampling")
    return math.pi * math.sqrt(x)


def kaiser_bessel_table(support: int, beta: float, per_cell: int = 1024) -> np.ndarray:
    """FP32 samples of the Kaiser-Bessel window at support * per_cell + 1 points spanning
    [-W/2, W/2] (both ends included; G is 1 at the centre)."""
    x = np.linspace(-0.5 * support, 0.5 * support, support * per_cell + 1)
    z = np.clip(1.0 - (2.0 * x / support) ** 2, 0.0, None)
    return (np.i0(beta * np.sqrt(z)) / np.i0(beta)).astype(np.float32)
