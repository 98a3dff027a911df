"""FP64 CPU oracle of the w-stacking imager (arXiv:2301.06061, section 2, Eq. 1-3).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library: the compiled part is ``wst_oracle.c`` (plain C, double
precision, OpenMP), built with gcc into ``liboracle.so`` next to it.

Parity status of every function is recorded in the module docstring of
``oracle.oracle``.
"""
from .oracle import (  # noqa: F401
    OracleConfig,
    build,
    degrid,
    degrid_on_grid,
    degrid_oversampled,
    dft_pixels,
    expand_rows,
    fft1d,
    fft2_centered,
    fold_w,
    gauss_legendre,
    grid,
    grid_config,
    image,
    image_on_grid,
    image_oversampled,
    image_pixels,
    kernel_eval,
    kernel_ft,
    kernel_grad,
    kernel_grad_on_grid,
    kernel_grad_oversampled,
    locate,
    n_minus_one,
    num_threads,
    plane_centre,
    predict_points,
    resolve_w_range,
)
