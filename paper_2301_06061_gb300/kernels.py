"""Tabulated convolution kernels for WST_KERNEL_TABLE (section 2, Eq. 3: the kernel is the
imager's free choice; the paper uses a Gaussian of 7 cells and names better kernels as
future work in its conclusions).

``kaiser_bessel_table``: the Kaiser-Bessel window G(x) = I0(beta sqrt(1 - (2x/W)^2)) /
I0(beta) on |x| <= W/2, sampled at ``per_cell`` points per cell (piecewise-linear between
samples, as the library interpolates every table).  ``kaiser_bessel_beta`` is the
shape parameter of Beatty, Nishimura & Pauly (IEEE TMI 24, 2005, Eq. 5) for a grid
oversampled by ``alpha``: beta = pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8).

``pswf_table``: the zeroth prolate spheroidal wave function G(x) = psi_0(c, 2x/W) /
psi_0(c, 0), the classical gridding kernel (the function on [-1, 1] whose Fourier
transform is most concentrated in |omega| <= c; Slepian and Pollak 1961).  It is computed
from that definition: psi_0 is the eigenfunction of the largest eigenvalue of the finite
Fourier transform, whose kernel on even functions is cos(c x t); the operator is
discretised with Gauss-Legendre quadrature, and psi_0 at any x follows from the
eigen-relation (Nystrom interpolation).  ``pswf_c`` puts the band edge of G,
c / (pi W) cycles per cell, at the first alias 1 - 1/(2 alpha) of the image's edge
frequency 1/(2 alpha) on a grid oversampled by alpha: c = pi W (1 - 1/(2 alpha)).

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


def pswf_c(support: int, alpha: float = 1.0) -> float:
    if alpha < 1.0:
        raise ValueError("oversampling below 1")
    return math.pi * support * (1.0 - 0.5 / alpha)


def pswf_values(c: float, x, n_quad: int = 0):
    """psi_0(c, x) for |x| <= 1, scaled to 1 at x = 0 (FP64)."""
    n = n_quad or max(64, int(2 * c) + 64)
    t, w = np.polynomial.legendre.leggauss(n)
    sw = np.sqrt(w)
    m = sw[:, None] * np.cos(c * np.outer(t, t)) * sw[None, :]  # symmetric: weights split
    lam, vec = np.linalg.eigh(m)
    psi_t = vec[:, -1] / sw  # the largest eigenvalue's eigenfunction at the nodes
    x = np.asarray(x, np.float64)
    psi_x = (np.cos(c * np.multiply.outer(x, t)) @ (w * psi_t)) / lam[-1]
    psi_0 = float((w * psi_t).sum() / lam[-1])
    return psi_x / psi_0


def pswf_table(support: int, c: float, per_cell: int = 1024) -> np.ndarray:
    """FP32 samples of psi_0(c, 2x/W) / psi_0(c, 0) at support * per_cell + 1 points
    spanning [-W/2, W/2] (both ends included)."""
    x = np.linspace(-0.5 * support, 0.5 * support, support * per_cell + 1)
    return pswf_values(c, 2.0 * x / support).astype(np.float32)
