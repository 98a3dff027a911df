"""The C-ABI library builds, loads and exports every entry point include/wst.h declares.

No compute call is made: this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wst_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_06061_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("wst_plan_create", "wst_grid", "wst_fft_correct", "wst_image", "wst_degrid",
                     "wst_kernel_grad", "wst_plan_set_vis"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2301_06061_gb300 import wst

    assert sorted(wst.EXPORTED) == declared_functions()
    for name in wst.EXPORTED:
        assert callable(getattr(wst, name))


def test_version_and_status_strings_without_gpu(lib):
    lib.wst_version.restype = ctypes.c_char_p
    lib.wst_status_string.restype = ctypes.c_char_p
    assert lib.wst_version().decode().count(".") == 2
    assert lib.wst_status_string(2).decode().startswith("out of memory")


def test_plan_create_rejects_bad_config_before_touching_the_device(lib):
    from paper_2301_06061_gb300 import wst

    lib = wst.load_library()
    bad = [wst.Config(n=100, fov=0.1, n_w=4), wst.Config(n=256, fov=-1.0, n_w=4),
           wst.Config(n=256, fov=0.1, n_w=0), wst.Config(n=256, fov=0.1, n_w=4, support=1),
           wst.Config(n=256, fov=0.1, n_w=4, kparam=0.0), wst.Config(n=32768, fov=0.1, n_w=4),
           wst.Config(n=256, fov=0.1, n_w=4, w_min=5.0, w_max=1.0)]
    for cfg in bad:
        h = ctypes.c_void_p()
        rc = lib.wst_plan_create(ctypes.byref(cfg.c()), None, ctypes.byref(h))
        assert rc in (1, 5) and not h.value


def _code_lines(path):
    """Source lines without comments (C/C++ // and /* */, Python #) or docstring prose."""
    text = open(path, encoding="utf-8").read()
    if path.endswith((".cu", ".cuh", ".c", ".h")):
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        return [ln.split("//")[0] for ln in text.splitlines()]
    text = re.sub(r'""".*?"""', "", text, flags=re.S)
    return [ln.split("#")[0] for ln in text.splitlines()]


def test_product_path_never_reaches_the_oracle():
    """The package and its CUDA sources neither import, load nor build anything under
    oracle/: the imager cannot fall back to the checker."""
    pkg = os.path.join(ROOT, "paper_2301_06061_gb300")
    files = [os.path.join(pkg, f) for f in os.listdir(pkg) if f.endswith(".py")]
    csrc = os.path.join(pkg, "csrc")
    files += [os.path.join(csrc, f) for f in os.listdir(csrc)]
    offenders = [(f, ln.strip()) for f in files for ln in _code_lines(f)
                 if re.search(r"\boracle\b|liboracle|wst_oracle", ln)]
    assert not offenders, offenders


def test_oracle_shares_no_code_with_the_cuda_library():
    """The oracle's C source includes only the C library, and its Python side loads only
    its own shared object."""
    src = open(os.path.join(ROOT, "oracle", "wst_oracle.c")).read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', src)
    assert set(includes) <= {"complex.h", "math.h", "stdint.h", "stdlib.h", "string.h", "omp.h", "stdio.h"}, includes
    for f in ("oracle.py", "__init__.py"):
        code = "\n".join(_code_lines(os.path.join(ROOT, "oracle", f)))
        assert "paper_2301_06061_gb300" not in code and "libwst" not in code and "csrc" not in code


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2301_06061_gb300 import wst

    monkeypatch.setattr(wst, "_lib", None)  # as in a fresh process
    with pytest.raises(RuntimeError, match="not found"):
        wst.load_library(str(tmp_path / "libwst.so"))


@pytest.mark.parametrize("change,status", [
    (dict(n=100), 5), (dict(n=32), 5), (dict(n=32768), 5), (dict(n=16384, oversample=2), 5),
    (dict(oversample=3), 5), (dict(fov=0.0), 1), (dict(fov=float("nan")), 1), (dict(n_w=0), 1),
    (dict(w_min=10.0, w_max=-10.0), 1), (dict(w_max=float("inf")), 1), (dict(support=1), 5),
    (dict(support=17), 5), (dict(kernel=7), 1), (dict(kparam=-1.0), 1), (dict(kernel=2, ktable_len=1), 1),
    (dict(flags=0x100), 1), (dict(batch=0), 1), (dict(planes_per_chunk=-1), 1),
    # an explicit grid side: a power of two in [N, 16384], N even and >= 64, not with oversample = 2
    (dict(n=200, grid_n=0), 5), (dict(n=200, grid_n=200), 5), (dict(n=200, grid_n=128), 5),
    (dict(n=201, grid_n=256), 5), (dict(n=48, grid_n=64), 5), (dict(n=10000, grid_n=32768), 5),
    (dict(grid_n=-256), 1), (dict(grid_n=512, oversample=2), 1),
])
def test_plan_create_rejects_invalid_configs_before_touching_the_device(lib, change, status):
    """Configuration errors come back as WST_ERR_INVALID_ARG (1) or WST_ERR_UNSUPPORTED
    (5) from host-side checks that run before any CUDA call (so this needs no GPU), and
    no plan is returned."""
    from paper_2301_06061_gb300 import wst

    fields = dict(n=256, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0, support=7, kernel=0, kparam=0.875,
                  ktable_len=0, flags=1, planes_per_chunk=0, batch=1, oversample=0, grid_n=0)
    fields.update(change)
    cfg = wst.wst_config(*[fields[name] for name, _ in wst.wst_config._fields_])
    h = ctypes.c_void_p(12345)
    fn = lib.wst_plan_create
    fn.argtypes = [ctypes.POINTER(wst.wst_config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    fn.restype = ctypes.c_int
    assert fn(ctypes.byref(cfg), None, ctypes.byref(h)) == status
    assert h.value is None
    assert fn(ctypes.byref(cfg), None, None) == 1  # no output handle


def test_every_entry_point_rejects_a_null_plan_or_bad_sizes_without_a_device(lib):
    """Argument errors are reported synchronously by host-side checks: a NULL plan, and
    sizes no call accepts.  Nothing here reaches the GPU."""
    from paper_2301_06061_gb300 import wst

    L = wst.load_library()
    calls = {
        "wst_plan_set_stream": (None, None),
        "wst_plan_set_wait_limit": (None, 0),
        "wst_plan_workspace_bytes": (None, 10, None),
        "wst_plan_set_workspace": (None, None, 0),
        "wst_plan_set_kernel_table": (None, None),
        "wst_plan_set_vis": (None, 0, None, None, None, None, None, None),
        "wst_plan_set_vis_rows": (None, 0, None, 0, None, 1, None, None, None),
        "wst_grid": (None, 0, 1, None),
        "wst_fft_correct": (None, 0, 1, None, None),
        "wst_correct": (None, None),
        "wst_image": (None, None, 0),
        "wst_image_range": (None, 0, 1, None, 0),
        "wst_degrid": (None, None, None, 0),
        "wst_kernel_grad": (None, None, None, 0),
        "wst_vis_cells": (None, None, None, None),
        "wst_get_stats": (None, None),
        "wst_dft": (1, None, None, None, None, None, 1, 0.1, 1, None, None, None, None),  # n < 2
        "wst_dft_noalloc": (1, None, None, None, None, None, 1, 0.1, 1, None, None, None, None),
        "wst_predict_points": (-1, None, None, None, 1, None, None, None, None, None),  # n_vis < 0
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == 1, name  # WST_ERR_INVALID_ARG
    L.wst_plan_destroy(None)  # a no-op
    assert L.wst_last_error(None) == b""
    for s in range(7):
        assert L.wst_status_string(s)
