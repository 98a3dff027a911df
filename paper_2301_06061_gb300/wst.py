"""Thin ctypes binding of ``libwst.so`` (declared in ``include/wst.h``).

Functions carry the C names and only marshal arguments: torch CUDA tensors are
passed as device pointers, the current torch stream as the CUDA stream.  Every
computation happens in the library's CUDA kernels; there is no CPU or PyTorch
fallback -- if the library cannot be loaded, every call raises.

``Plan`` bundles a plan handle with a torch-allocated workspace for convenience.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwst.so")

WST_OK = 0
STATUS = {0: "WST_OK", 1: "WST_ERR_INVALID_ARG", 2: "WST_ERR_OOM", 3: "WST_ERR_CUDA",
          4: "WST_ERR_TIMEOUT", 5: "WST_ERR_UNSUPPORTED", 6: "WST_ERR_STATE"}

WST_KERNEL_GAUSS, WST_KERNEL_ES, WST_KERNEL_TABLE = 0, 1, 2
WST_FLAG_KAHAN, WST_FLAG_FP64_SCREEN, WST_FLAG_TIMING, WST_FLAG_WFOLD = 0x1, 0x2, 0x4, 0x8
WST_NO_CORRECTION = 0x1

EXPORTED = [
    "wst_version", "wst_status_string", "wst_plan_create", "wst_plan_destroy", "wst_plan_set_stream",
    "wst_plan_set_wait_limit", "wst_plan_workspace_bytes", "wst_plan_set_workspace", "wst_plan_set_kernel_table",
    "wst_plan_set_vis", "wst_plan_set_vis_rows", "wst_grid", "wst_fft_correct", "wst_correct", "wst_image", "wst_image_range", "wst_degrid",
    "wst_kernel_grad", "wst_vis_cells", "wst_get_stats", "wst_last_error", "wst_dft",
    "wst_predict_points", "wst_dft_noalloc",
]


class WstError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class wst_config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("fov", ctypes.c_double),
        ("n_w", ctypes.c_int32),
        ("w_min", ctypes.c_double),
        ("w_max", ctypes.c_double),
        ("support", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("kparam", ctypes.c_double),
        ("ktable_len", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("planes_per_chunk", ctypes.c_int32),
        ("batch", ctypes.c_int32),
        ("oversample", ctypes.c_int32),
        ("grid_n", ctypes.c_int32),
    ]


class wst_stats(ctypes.Structure):
    _fields_ = [
        ("n_vis", ctypes.c_int64),
        ("n_kept", ctypes.c_int64),
        ("n_dropped", ctypes.c_int64),
        ("n_nonfinite", ctypes.c_int64),
        ("w_min", ctypes.c_double),
        ("w_max", ctypes.c_double),
        ("ms_sort", ctypes.c_float),
        ("ms_grid", ctypes.c_float),
        ("ms_rows", ctypes.c_float),
        ("ms_cols_a", ctypes.c_float),
        ("ms_cols_b", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("device_error", ctypes.c_int32),
        ("n_chunks", ctypes.c_int32),
        ("n_launches", ctypes.c_int64),
        ("n_rows_gridded", ctypes.c_int64),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libwst.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} not found: build it with paper_2301_06061_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, I32, I64, U32, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        sig = {
            "wst_version": ([], ctypes.c_char_p),
            "wst_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "wst_plan_create": ([ctypes.POINTER(wst_config), P, ctypes.POINTER(P)], ctypes.c_int),
            "wst_plan_destroy": ([P], None),
            "wst_plan_set_stream": ([P, P], ctypes.c_int),
            "wst_plan_set_wait_limit": ([P, ctypes.c_uint64], ctypes.c_int),
            "wst_plan_workspace_bytes": ([P, I64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
            "wst_plan_set_workspace": ([P, P, ctypes.c_size_t], ctypes.c_int),
            "wst_plan_set_kernel_table": ([P, P], ctypes.c_int),
            "wst_plan_set_vis": ([P, I64, P, P, P, P, P, P], ctypes.c_int),
            "wst_plan_set_vis_rows": ([P, I64, P, I64, P, I32, P, P, P], ctypes.c_int),
            "wst_grid": ([P, I32, I32, P], ctypes.c_int),
            "wst_fft_correct": ([P, I32, I32, P, P], ctypes.c_int),
            "wst_correct": ([P, P], ctypes.c_int),
            "wst_image": ([P, P, U32], ctypes.c_int),
            "wst_image_range": ([P, I32, I32, P, U32], ctypes.c_int),
            "wst_degrid": ([P, P, P, U32], ctypes.c_int),
            "wst_kernel_grad": ([P, P, P, U32], ctypes.c_int),
            "wst_vis_cells": ([P, P, P, P], ctypes.c_int),
            "wst_get_stats": ([P, ctypes.POINTER(wst_stats)], ctypes.c_int),
            "wst_last_error": ([P], ctypes.c_char_p),
            "wst_dft": ([I64, P, P, P, P, P, I32, D, I64, P, P, P, P], ctypes.c_int),
            "wst_predict_points": ([I64, P, P, P, I64, P, P, P, P, P], ctypes.c_int),
            "wst_dft_noalloc": ([I64, P, P, P, P, P, I32, D, I64, P, P, P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _ptr(t, host_ok: bool = False):
    """Device pointer of a CUDA tensor; with host_ok, also a page-locked CPU tensor (the
    entry points that accept host memory read or write it in place)."""
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda and not (host_ok and t.is_pinned()):
            raise ValueError("libwst takes CUDA tensors" + (" or pinned CPU tensors" if host_ok else ""))
        if not t.is_contiguous():
            raise ValueError("libwst takes contiguous tensors")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(status: int, where: str, plan=None):
    if status != WST_OK:
        detail = ""
        if plan is not None:
            msg = load_library().wst_last_error(plan)
            detail = msg.decode() if msg else ""
        raise WstError(status, where, detail)


# ----------------------------------------------------------------------------------------
# the C entry points, one Python function each (argument marshalling only)
# ----------------------------------------------------------------------------------------

def wst_version() -> str:
    return load_library().wst_version().decode()


def wst_status_string(status: int) -> str:
    return load_library().wst_status_string(int(status)).decode()


def wst_plan_create(cfg: wst_config, stream=None):
    h = ctypes.c_void_p()
    _check(load_library().wst_plan_create(ctypes.byref(cfg), _stream(stream), ctypes.byref(h)),
           "wst_plan_create")
    return h


def wst_plan_destroy(plan) -> None:
    load_library().wst_plan_destroy(plan)


def wst_plan_set_stream(plan, stream=None) -> None:
    _check(load_library().wst_plan_set_stream(plan, _stream(stream)), "wst_plan_set_stream", plan)


def wst_plan_set_wait_limit(plan, wait_ns: int) -> None:
    _check(load_library().wst_plan_set_wait_limit(plan, int(wait_ns)), "wst_plan_set_wait_limit", plan)


def wst_plan_workspace_bytes(plan, n_vis: int) -> int:
    out = ctypes.c_size_t()
    _check(load_library().wst_plan_workspace_bytes(plan, int(n_vis), ctypes.byref(out)),
           "wst_plan_workspace_bytes", plan)
    return int(out.value)


def wst_plan_set_workspace(plan, buf: torch.Tensor) -> None:
    _check(load_library().wst_plan_set_workspace(plan, _ptr(buf), buf.numel() * buf.element_size()),
           "wst_plan_set_workspace", plan)


def wst_plan_set_kernel_table(plan, table: torch.Tensor) -> None:
    assert table.dtype == torch.float32
    _check(load_library().wst_plan_set_kernel_table(plan, _ptr(table)), "wst_plan_set_kernel_table", plan)


def wst_plan_set_vis(plan, u, v, w, vis, weight=None, batch_offsets=None) -> None:
    n = u.numel()
    for t in (u, v, w):
        assert t.dtype == torch.float32 and t.numel() == n
    assert vis.dtype == torch.complex64 and vis.numel() == n
    if weight is not None:
        assert weight.dtype == torch.float32 and weight.numel() == n
    off = None
    if batch_offsets is not None:
        arr = (ctypes.c_int64 * len(batch_offsets))(*[int(x) for x in batch_offsets])
        off = ctypes.cast(arr, ctypes.c_void_p)
    h = True  # device tensors or pinned host tensors
    _check(load_library().wst_plan_set_vis(plan, n, _ptr(u, h), _ptr(v, h), _ptr(w, h), _ptr(vis, h),
                                           _ptr(weight, h), off),
           "wst_plan_set_vis", plan)


def wst_plan_set_vis_rows(plan, uvw_m, chan_scale, vis, weight=None, batch_offsets=None) -> None:
    """Visibility i = row (i // n_chan), channel (i % n_chan); uvw_m FP64 [n_rows, 3] metres,
    chan_scale FP64 [n_chan] (nu / c), vis complex64 [n_vis] with n_vis <= n_rows * n_chan."""
    n = vis.numel()
    assert uvw_m.dtype == torch.float64 and uvw_m.dim() == 2 and uvw_m.shape[1] == 3
    assert chan_scale.dtype == torch.float64 and chan_scale.dim() == 1
    assert vis.dtype == torch.complex64
    if weight is not None:
        assert weight.dtype == torch.float32 and weight.numel() == n
    off = None
    if batch_offsets is not None:
        arr = (ctypes.c_int64 * len(batch_offsets))(*[int(x) for x in batch_offsets])
        off = ctypes.cast(arr, ctypes.c_void_p)
    h = True  # device tensors or pinned host tensors
    _check(load_library().wst_plan_set_vis_rows(plan, n, _ptr(uvw_m, h), uvw_m.shape[0], _ptr(chan_scale, h),
                                                chan_scale.numel(), _ptr(vis, h), _ptr(weight, h), off),
           "wst_plan_set_vis_rows", plan)


def wst_grid(plan, plane_begin: int, plane_end: int, grid_out: torch.Tensor) -> None:
    assert grid_out.dtype == torch.complex64
    _check(load_library().wst_grid(plan, plane_begin, plane_end, _ptr(grid_out)), "wst_grid", plan)


def wst_fft_correct(plan, plane_begin: int, plane_end: int, grid_inout, image_inout) -> None:
    _check(load_library().wst_fft_correct(plan, plane_begin, plane_end, _ptr(grid_inout), _ptr(image_inout)),
           "wst_fft_correct", plan)


def wst_correct(plan, image_inout) -> None:
    _check(load_library().wst_correct(plan, _ptr(image_inout)), "wst_correct", plan)


def wst_image(plan, image_out: torch.Tensor, flags: int = 0) -> None:
    assert image_out.dtype == torch.complex64
    _check(load_library().wst_image(plan, _ptr(image_out, True), flags), "wst_image", plan)


def wst_image_range(plan, plane_begin: int, plane_end: int, image_out: torch.Tensor, flags: int = 0) -> None:
    assert image_out.dtype == torch.complex64
    _check(load_library().wst_image_range(plan, int(plane_begin), int(plane_end), _ptr(image_out, True), flags),
           "wst_image_range", plan)


def wst_degrid(plan, dimage: torch.Tensor, dvis_out: torch.Tensor, flags: int = 0) -> None:
    assert dimage.dtype == torch.complex64 and dvis_out.dtype == torch.complex64
    _check(load_library().wst_degrid(plan, _ptr(dimage), _ptr(dvis_out), flags), "wst_degrid", plan)


def wst_kernel_grad(plan, dimage: torch.Tensor, dtable_out: torch.Tensor, flags: int = WST_NO_CORRECTION) -> None:
    _check(load_library().wst_kernel_grad(plan, _ptr(dimage), _ptr(dtable_out), flags), "wst_kernel_grad", plan)


def wst_vis_cells(plan, plane_out, i0_out, j0_out) -> None:
    _check(load_library().wst_vis_cells(plan, _ptr(plane_out), _ptr(i0_out), _ptr(j0_out)), "wst_vis_cells", plan)


def wst_get_stats(plan) -> dict:
    st = wst_stats()
    rc = load_library().wst_get_stats(plan, ctypes.byref(st))
    if rc not in (WST_OK, 4):
        _check(rc, "wst_get_stats", plan)
    return {name: getattr(st, name) for name, _ in wst_stats._fields_}


def wst_last_error(plan) -> str:
    msg = load_library().wst_last_error(plan)
    return msg.decode() if msg else ""


def wst_dft(u, v, w, vis, n: int, fov: float, pa, pb, out, weight=None, stream=None) -> None:
    _check(load_library().wst_dft(u.numel(), _ptr(u), _ptr(v), _ptr(w), _ptr(vis), _ptr(weight), int(n),
                                  float(fov), pa.numel(), _ptr(pa), _ptr(pb), _ptr(out), _stream(stream)),
           "wst_dft")


WST_DFT_NOALLOC_MAX_PIX = 4096


def wst_dft_noalloc(u, v, w, vis, n: int, fov: float, pa, pb, out, weight=None, stream=None) -> int:
    """Allocation-free direct transform; returns the status (raises on CUDA errors only)."""
    rc = load_library().wst_dft_noalloc(u.numel(), _ptr(u), _ptr(v), _ptr(w), _ptr(vis), _ptr(weight), int(n),
                                        float(fov), pa.numel(), _ptr(pa), _ptr(pb), _ptr(out), _stream(stream))
    if rc == 3:
        _check(rc, "wst_dft_noalloc")
    return rc


def wst_predict_points(u, v, w, l, m, flux, out, stream=None) -> None:
    _check(load_library().wst_predict_points(u.numel(), _ptr(u), _ptr(v), _ptr(w), l.numel(), _ptr(l), _ptr(m),
                                             _ptr(flux), _ptr(out), _stream(stream)),
           "wst_predict_points")


# ----------------------------------------------------------------------------------------
# convenience: a plan with its workspace
# ----------------------------------------------------------------------------------------

@dataclass
class Config:
    n: int
    fov: float
    n_w: int
    w_min: float = 0.0
    w_max: float = 0.0
    support: int = 7
    kernel: int = WST_KERNEL_GAUSS
    kparam: float = 0.875
    ktable_len: int = 0
    flags: int = WST_FLAG_KAHAN
    planes_per_chunk: int = 0
    batch: int = 1
    oversample: int = 0
    grid_n: int = 0  # grid side M (a power of two >= n); 0: n, or 2n with oversample = 2

    def c(self) -> wst_config:
        return wst_config(self.n, self.fov, self.n_w, self.w_min, self.w_max, self.support, self.kernel,
                          self.kparam, self.ktable_len, self.flags, self.planes_per_chunk, self.batch,
                          self.oversample, self.grid_n)


DEFAULT_SIGMA = {7: 0.875, 8: 0.925}


class Plan:
    """A wst plan plus a torch-allocated workspace sized for the visibilities it sees."""

    def __init__(self, cfg: Config, device=None):
        self.cfg = cfg
        self.device = torch.device("cuda") if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.handle = wst_plan_create(cfg.c())
        self.ws = None
        self.n_vis = 0
        # bumped by every call that rebinds the visibilities or the kernel table, so that
        # a caller holding work from an earlier binding can tell the plan has moved on
        self.generation = 0

    def close(self):
        if self.handle is not None:
            wst_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ensure_workspace(self, n_vis: int):
        need = wst_plan_workspace_bytes(self.handle, n_vis)
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            wst_plan_set_workspace(self.handle, self.ws)

    def set_kernel_table(self, table: torch.Tensor):
        wst_plan_set_kernel_table(self.handle, table.contiguous())
        self.generation += 1

    def set_vis(self, u, v, w, vis, weight=None, batch_offsets=None):
        self.ensure_workspace(u.numel())
        wst_plan_stream(self.handle)
        wst_plan_set_vis(self.handle, u, v, w, vis, weight, batch_offsets)
        self.n_vis = u.numel()
        self.generation += 1

    def set_vis_rows(self, uvw_m, chan_scale, vis, weight=None, batch_offsets=None):
        self.ensure_workspace(vis.numel())
        wst_plan_stream(self.handle)
        wst_plan_set_vis_rows(self.handle, uvw_m, chan_scale, vis, weight, batch_offsets)
        self.n_vis = vis.numel()
        self.generation += 1

    def image(self, out=None, flags: int = 0) -> torch.Tensor:
        c = self.cfg
        if out is None:
            out = torch.empty((c.batch, c.n, c.n), dtype=torch.complex64, device=self.device)
        wst_plan_stream(self.handle)
        wst_image(self.handle, out, flags)
        return out

    def image_range(self, plane_begin: int, plane_end: int, out=None, flags: int = 0) -> torch.Tensor:
        """The partial image of global planes [plane_begin, plane_end) (wst_image_range)."""
        c = self.cfg
        if out is None:
            out = torch.empty((c.batch, c.n, c.n), dtype=torch.complex64, device=self.device)
        wst_plan_stream(self.handle)
        wst_image_range(self.handle, plane_begin, plane_end, out, flags)
        return out

    def degrid(self, dimage, out=None, flags: int = 0) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n_vis, dtype=torch.complex64, device=self.device)
        wst_plan_stream(self.handle)
        wst_degrid(self.handle, dimage.contiguous(), out, flags)
        return out

    def kernel_grad(self, dimage, out=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.cfg.ktable_len, dtype=torch.float32, device=self.device)
        wst_plan_stream(self.handle)
        wst_kernel_grad(self.handle, dimage.contiguous(), out, WST_NO_CORRECTION)
        return out

    def stats(self) -> dict:
        return wst_get_stats(self.handle)


def wst_plan_stream(plan) -> None:
    """Point the plan at torch's current stream (calls enqueue there)."""
    wst_plan_set_stream(plan, None)
