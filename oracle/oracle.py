"""ctypes wrapper of the FP64 oracle (``wst_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every function follows a passage of arXiv:2301.06061:

* ``locate``        -- nearest w-plane and kernel footprint (section 2, Eq. 3)
* ``grid``          -- convolutional gridding (Eq. 3)
* ``fft2_centered`` -- per-plane 2D Fourier transform (Eq. 2, inner integral)
* ``image``         -- full w-stacking image (Eq. 2): grid, transform, phase screen,
                       sum over planes, grid correction
* ``image_pixels``  -- the same image evaluated pixel by pixel without planes
* ``dft_pixels``    -- direct transform, the exact dirty image (conjugate of Eq. 1)
* ``predict_points``-- Eq. 1 for a point-source sky (test input synthesis only)
* ``degrid``        -- adjoint of ``image`` (degridding; listed as future work in
                       the paper's conclusions)
* ``kernel_grad``   -- gradient of a real loss w.r.t. a tabulated kernel
* ``kernel_ft``     -- Ghat(nu), the Fourier transform of the truncated kernel
* ``fold_w``        -- the w-folding variant's Hermitian mirror of w < 0 visibilities
                       (not in the paper; applied to the inputs of the functions above)
* ``image_on_grid`` -- the oversampled-grid variant (not in the paper): ``image``
                       on a grid of M cells (a power of two, M >= N; ``grid_config``),
                       cropped to the central N x N (N even, any size), oversampling
                       factor M/N; ``image_oversampled`` is the case M = 2N
* ``degrid_on_grid``, ``kernel_grad_on_grid`` (and the ``_oversampled`` M = 2N cases)
                    -- its adjoint and kernel gradient: the image zero-padded to the
                       grid (the adjoint of the crop), then ``degrid`` / ``kernel_grad``
                       on the grid
* ``expand_rows``   -- per-visibility (u, v, w) in wavelengths from per-row baseline
                       coordinates in metres and per-channel nu / c (the layout of
                       the LOFAR datasets of section 4; input expansion only)

Pins (tests/test_oracle_*.py) tie each one to something other than itself:
numpy/pocketfft and the textbook DFT for the FFT; closed forms for Ghat and the
screen; brute-force DFT within the analytic aliasing bound for the image;
linearity, Hermitian symmetry and the single-visibility flat image; the
dot-product identity for the adjoint; finite differences for the kernel
gradient; exact integer placement rules for ``locate``; for ``fold_w``, the
invariance of the real part of the direct transform; for ``image_on_grid``, the
direct transform within the aliasing bound of the frequencies |nu| <= N/(2M) the image
keeps (M = 2N, and M/N = 1.28 and 1.51 with N not a power of two); for
``degrid_on_grid``, the dot-product identity with ``image_on_grid``; for
``kernel_grad_on_grid``, central differences of ``image_on_grid``; for
``expand_rows``, exactly representable products, the (row, channel) order with a
partial last row, and a product whose one rounding differs from rounding its factors
first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wst_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

KERNELS = {"gauss": 0, "es": 1, "table": 2}


def build(force: bool = False) -> str:
    """Compile ``wst_oracle.c`` with gcc (double precision, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("fov", ctypes.c_double),
        ("n_w", ctypes.c_int32),
        ("w_min", ctypes.c_double),
        ("w_max", ctypes.c_double),
        ("support", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("kparam", ctypes.c_double),
        ("ktable", ctypes.POINTER(ctypes.c_double)),
        ("ktable_len", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def _declare(lib):
    cfgp = ctypes.POINTER(_Cfg)
    lib.wo_kernel_eval.argtypes = [cfgp, ctypes.c_double]
    lib.wo_kernel_eval.restype = ctypes.c_double
    lib.wo_gauss_legendre.argtypes = [ctypes.c_int, _P, _P]
    lib.wo_kernel_ft.argtypes = [cfgp, _I64, _P, _P]
    lib.wo_locate.argtypes = [cfgp, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    lib.wo_locate.restype = _I64
    lib.wo_grid.argtypes = [cfgp, _I64, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]
    lib.wo_fft1d.argtypes = [_P, _I64, ctypes.c_int]
    lib.wo_fft2_centered.argtypes = [_P, _I64, ctypes.c_int]
    lib.wo_n_minus_one.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.wo_n_minus_one.restype = ctypes.c_double
    lib.wo_plane_centre.argtypes = [cfgp, ctypes.c_int]
    lib.wo_plane_centre.restype = ctypes.c_double
    lib.wo_image.argtypes = [cfgp, _I64, _P, _P, _P, _P, _P, ctypes.c_int, _P]
    lib.wo_image_pixels.argtypes = [cfgp, _I64, _P, _P, _P, _P, _P, ctypes.c_int, _I64, _P, _P, _P]
    lib.wo_dft_pixels.argtypes = [_I64, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double,
                                  _I64, _P, _P, _P]
    lib.wo_predict_points.argtypes = [_I64, _P, _P, _P, _I64, _P, _P, _P, _P]
    lib.wo_degrid.argtypes = [cfgp, _I64, _P, _P, _P, _P, _P, ctypes.c_int, _P, _P]
    lib.wo_kernel_grad.argtypes = [cfgp, _I64, _P, _P, _P, _P, _P, _P, _P]
    lib.wo_num_threads.restype = ctypes.c_int


@dataclass
class OracleConfig:
    """Imaging configuration as the oracle reads it (w range already resolved)."""

    n: int
    fov: float
    n_w: int
    w_min: float
    w_max: float
    support: int = 7
    kernel: str = "gauss"
    kparam: float = 0.875
    ktable: np.ndarray | None = None

    def _c(self):
        cfg = _Cfg()
        cfg.n = int(self.n)
        cfg.fov = float(self.fov)
        cfg.n_w = int(self.n_w)
        cfg.w_min = float(self.w_min)
        cfg.w_max = float(self.w_max)
        cfg.support = int(self.support)
        cfg.kernel = KERNELS[self.kernel]
        cfg.kparam = float(self.kparam)
        if self.kernel == "table":
            tab = np.ascontiguousarray(self.ktable, dtype=np.float64)
            self._tab_keep = tab
            cfg.ktable = tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            cfg.ktable_len = int(tab.size)
        else:
            cfg.ktable = None
            cfg.ktable_len = 0
        self._cfg_keep = cfg
        return ctypes.byref(cfg)


def fold_w(u, v, w, vis):
    """The w-folding variant (not in the paper): every visibility with w < 0 replaced by
    its Hermitian mirror (-u, -v, -w, conj V).  The mirrored term of the dirty image is
    the complex conjugate of the original one, so the real part of the image is
    unchanged.  Sign flips are exact in FP32; non-finite w are left alone."""
    u, v, w = (np.array(a, dtype=np.float32, copy=True) for a in (u, v, w))
    vis = np.array(vis, dtype=np.complex64, copy=True)
    m = w < 0
    u[m], v[m], w[m] = -u[m], -v[m], -w[m]
    vis[m] = np.conj(vis[m])
    return u, v, w, vis


def expand_rows(uvw_m, chan_scale, n_vis: int):
    """Coordinates of visibilities stored by row (one baseline at one time) and channel,
    as in the LOFAR datasets of section 4: visibility i is row i // C, channel i % C
    (C channels), at (u, v, w) = baseline (metres) x nu_c / c in wavelengths, the
    product taken in FP64 and rounded once to FP32."""
    uvw_m = np.asarray(uvw_m, dtype=np.float64).reshape(-1, 3)
    scale = np.asarray(chan_scale, dtype=np.float64).reshape(-1)
    if n_vis > uvw_m.shape[0] * scale.size:
        raise ValueError("n_vis exceeds rows x channels")
    i = np.arange(int(n_vis))
    row, ch = i // scale.size, i % scale.size
    return tuple((uvw_m[row, k] * scale[ch]).astype(np.float32) for k in range(3))


def resolve_w_range(w: np.ndarray, w_min: float, w_max: float) -> tuple[float, float]:
    """Plane range: the configured one, or the min/max of the finite w when equal."""
    if w_min != w_max:
        return float(w_min), float(w_max)
    wf = np.asarray(w, dtype=np.float32)
    wf = wf[np.isfinite(wf)]
    if wf.size == 0:
        return 0.0, 0.0
    return float(wf.min()), float(wf.max())


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _vis(v):
    v = np.ascontiguousarray(v, dtype=np.complex64)
    return v.view(np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _inputs(u, v, w, vis, weight):
    u, v, w = _f32(u), _f32(v), _f32(w)
    visf = _vis(vis)
    wt = None if weight is None else _f32(weight)
    return u, v, w, visf, wt


def num_threads() -> int:
    return int(_load().wo_num_threads())


def kernel_eval(cfg: OracleConfig, x: float) -> float:
    return float(_load().wo_kernel_eval(cfg._c(), float(x)))


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().wo_gauss_legendre(n, x.ctypes.data, w.ctypes.data)
    return x, w


def kernel_ft(cfg: OracleConfig, nu) -> np.ndarray:
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    out = np.zeros_like(nu)
    _load().wo_kernel_ft(cfg._c(), nu.size, nu.ctypes.data, out.ctypes.data)
    return out


def locate(cfg: OracleConfig, u, v, w, vis, weight=None):
    """Per visibility (plane k, tap start i0 along u, tap start j0 along v, status).

    status: 0 kept, 1 dropped (footprint leaves the grid), 2 non-finite input.
    """
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    n = u.size
    k = np.empty(n, np.int32)
    i0 = np.empty(n, np.int32)
    j0 = np.empty(n, np.int32)
    st = np.empty(n, np.int32)
    _load().wo_locate(cfg._c(), n, u.ctypes.data, v.ctypes.data, w.ctypes.data, visf.ctypes.data,
                      _ptr(wt), k.ctypes.data, i0.ctypes.data, j0.ctypes.data, st.ctypes.data)
    return k, i0, j0, st


def grid(cfg: OracleConfig, u, v, w, vis, weight=None, k0: int = 0, k1: int | None = None):
    """Gridded planes [k0, k1) as complex128 array (k1-k0, N, N), row index = v cell."""
    k1 = cfg.n_w if k1 is None else k1
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    out = np.zeros((k1 - k0, cfg.n, cfg.n), np.complex128)
    _load().wo_grid(cfg._c(), u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data, visf.ctypes.data,
                    _ptr(wt), k0, k1, out.ctypes.data)
    return out


def fft1d(x, sign: int = +1) -> np.ndarray:
    x = np.array(x, dtype=np.complex128, copy=True)
    _load().wo_fft1d(x.ctypes.data, x.size, int(sign))
    return x


def fft2_centered(g, sign: int = +1) -> np.ndarray:
    g = np.array(g, dtype=np.complex128, copy=True, order="C")
    _load().wo_fft2_centered(g.ctypes.data, g.shape[0], int(sign))
    return g


def n_minus_one(l: float, m: float) -> float:
    return float(_load().wo_n_minus_one(float(l), float(m)))


def plane_centre(cfg: OracleConfig, k: int) -> float:
    return float(_load().wo_plane_centre(cfg._c(), int(k)))


def image(cfg: OracleConfig, u, v, w, vis, weight=None, correct: bool = True) -> np.ndarray:
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    out = np.zeros((cfg.n, cfg.n), np.complex128)
    _load().wo_image(cfg._c(), u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data,
                     visf.ctypes.data, _ptr(wt), int(bool(correct)), out.ctypes.data)
    return out


def grid_config(cfg: OracleConfig, m: int) -> OracleConfig:
    """The configuration of an m-cell grid (m a power of two, m >= n) with the pixels of
    ``cfg``: cells of n/(m fov) wavelengths, i.e. a field of fov m / n computed as
    (fov m) / n, one rounding (the order the library uses, so that placement decisions
    agree bit for bit)."""
    n = int(cfg.n)
    if m < n or m & (m - 1):
        raise ValueError("the grid side must be a power of two no smaller than the image")
    return OracleConfig(m, cfg.fov * m / n, cfg.n_w, cfg.w_min, cfg.w_max, cfg.support,
                        cfg.kernel, cfg.kparam, cfg.ktable)


def _crop_offset(n: int, m: int) -> int:
    if n % 2:
        raise ValueError("an image cropped from a larger grid has an even side")
    return (m - n) // 2


def image_on_grid(cfg: OracleConfig, m: int, u, v, w, vis, weight=None, correct: bool = True) -> np.ndarray:
    """The oversampled-grid variant (not in the paper): the image of ``cfg`` (n pixels of
    fov/n, n even, any size) as the central n x n of the plain algorithm run on a grid of
    m cells (``grid_config``): the same pixels, a wider transform, oversampling factor
    m/n.  Grid pixel a + c, c = (m - n)/2, is image pixel a: both sit at
    (a - n/2) fov/n."""
    n = int(cfg.n)
    c = _crop_offset(n, m)
    full = image(grid_config(cfg, m), u, v, w, vis, weight, correct)
    return full[c:c + n, c:c + n].copy()


def image_oversampled(cfg: OracleConfig, oversample: int, u, v, w, vis, weight=None,
                      correct: bool = True) -> np.ndarray:
    """``image_on_grid`` with m = oversample * n."""
    return image_on_grid(cfg, oversample * int(cfg.n), u, v, w, vis, weight, correct)


def _zero_pad(dimage, n: int, m: int) -> np.ndarray:
    """The n x n image in the centre of a zero m x m grid image: the adjoint of the centre
    crop of ``image_on_grid``."""
    big = np.zeros((m, m), np.complex128)
    c = _crop_offset(n, m)
    big[c:c + n, c:c + n] = np.asarray(dimage, np.complex128).reshape(n, n)
    return big


def degrid_on_grid(cfg: OracleConfig, m: int, u, v, w, vis, dimage, weight=None, correct: bool = True) -> np.ndarray:
    """Adjoint of ``image_on_grid``: the image is zero-padded to the m x m grid (the
    adjoint of the crop) and degridded by ``degrid`` on that grid."""
    return degrid(grid_config(cfg, m), u, v, w, vis, _zero_pad(dimage, int(cfg.n), m), weight, correct)


def kernel_grad_on_grid(cfg: OracleConfig, m: int, u, v, w, vis, dimage, weight=None) -> np.ndarray:
    """Gradient of Re<dimage, U> w.r.t. the kernel table, U the uncorrected
    ``image_on_grid``: ``kernel_grad`` on the grid with the zero-padded dimage."""
    return kernel_grad(grid_config(cfg, m), u, v, w, vis, _zero_pad(dimage, int(cfg.n), m), weight)


def degrid_oversampled(cfg: OracleConfig, oversample: int, u, v, w, vis, dimage, weight=None,
                       correct: bool = True) -> np.ndarray:
    """``degrid_on_grid`` with m = oversample * n."""
    return degrid_on_grid(cfg, oversample * int(cfg.n), u, v, w, vis, dimage, weight, correct)


def kernel_grad_oversampled(cfg: OracleConfig, oversample: int, u, v, w, vis, dimage, weight=None) -> np.ndarray:
    """``kernel_grad_on_grid`` with m = oversample * n."""
    return kernel_grad_on_grid(cfg, oversample * int(cfg.n), u, v, w, vis, dimage, weight)


def image_pixels(cfg: OracleConfig, u, v, w, vis, pa, pb, weight=None,
                 correct: bool = True) -> np.ndarray:
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    pa = np.ascontiguousarray(pa, np.int32)
    pb = np.ascontiguousarray(pb, np.int32)
    out = np.zeros(pa.size, np.complex128)
    _load().wo_image_pixels(cfg._c(), u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data,
                            visf.ctypes.data, _ptr(wt), int(bool(correct)), pa.size,
                            pa.ctypes.data, pb.ctypes.data, out.ctypes.data)
    return out


def dft_pixels(u, v, w, vis, n: int, fov: float, pa, pb, weight=None) -> np.ndarray:
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    pa = np.ascontiguousarray(pa, np.int32)
    pb = np.ascontiguousarray(pb, np.int32)
    out = np.zeros(pa.size, np.complex128)
    _load().wo_dft_pixels(u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data, visf.ctypes.data,
                          _ptr(wt), int(n), float(fov), pa.size, pa.ctypes.data, pb.ctypes.data,
                          out.ctypes.data)
    return out


def predict_points(u, v, w, l, m, flux) -> np.ndarray:
    u, v, w = _f32(u), _f32(v), _f32(w)
    l = np.ascontiguousarray(l, np.float64)
    m = np.ascontiguousarray(m, np.float64)
    flux = np.ascontiguousarray(flux, np.float64)
    out = np.zeros(u.size, np.complex128)
    _load().wo_predict_points(u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data, l.size,
                              l.ctypes.data, m.ctypes.data, flux.ctypes.data, out.ctypes.data)
    return out


def degrid(cfg: OracleConfig, u, v, w, vis, dimage, weight=None, correct: bool = True) -> np.ndarray:
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    d = np.ascontiguousarray(dimage, np.complex128)
    out = np.zeros(u.size, np.complex128)
    _load().wo_degrid(cfg._c(), u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data,
                      visf.ctypes.data, _ptr(wt), int(bool(correct)), d.ctypes.data,
                      out.ctypes.data)
    return out


def kernel_grad(cfg: OracleConfig, u, v, w, vis, dimage, weight=None) -> np.ndarray:
    assert cfg.kernel == "table"
    u, v, w, visf, wt = _inputs(u, v, w, vis, weight)
    d = np.ascontiguousarray(dimage, np.complex128)
    out = np.zeros(len(cfg.ktable), np.float64)
    _load().wo_kernel_grad(cfg._c(), u.size, u.ctypes.data, v.ctypes.data, w.ctypes.data,
                           visf.ctypes.data, _ptr(wt), d.ctypes.data, out.ctypes.data)
    return out
