"""torch.autograd bindings of the imager and of its tabulated kernel.

``ImageFn``: D = A V, forward ``wst_image``, backward ``wst_degrid``.  A is C-linear
in the visibilities, so the vector-Jacobian product torch asks for is the adjoint
A^H applied to the incoming gradient (degridding; the paper's conclusions list it
as the next step).  Both directions run in libwst's CUDA kernels.

``KernelImageFn``: U(table), the image without grid correction as a function of a
tabulated kernel's samples; backward ``wst_kernel_grad``.  The grid correction,
which also depends on the table, is left to differentiable torch code
(``learned.correction_from_table``).
"""
from __future__ import annotations

import torch

from . import wst


class ImageFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vis, plan, u, v, w, weight, flags):
        plan.set_vis(u, v, w, vis.detach().to(torch.complex64).contiguous(), weight)
        out = plan.image(flags=flags)
        ctx.plan = plan
        ctx.flags = flags
        ctx.in_dtype = vis.dtype
        return out if vis.dtype == torch.complex64 else out.to(vis.dtype)

    @staticmethod
    def backward(ctx, grad):
        g = grad.detach().to(torch.complex64).contiguous()
        dvis = ctx.plan.degrid(g, flags=ctx.flags)
        return dvis.to(ctx.in_dtype), None, None, None, None, None, None


def image(vis, plan, u, v, w, weight=None, flags: int = 0):
    """Differentiable w-stacking image of ``vis`` (complex) on a ``wst.Plan``."""
    return ImageFn.apply(vis, plan, u, v, w, weight, flags)


class KernelImageFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, table, plan, u, v, w, vis, weight):
        plan.set_kernel_table(table.detach().to(torch.float32).contiguous())
        plan.set_vis(u, v, w, vis, weight)
        out = plan.image(flags=wst.WST_NO_CORRECTION)
        ctx.plan = plan
        return out

    @staticmethod
    def backward(ctx, grad):
        dtab = ctx.plan.kernel_grad(grad.detach().to(torch.complex64).contiguous())
        return dtab, None, None, None, None, None, None


def kernel_image(table, plan, u, v, w, vis, weight=None):
    """Uncorrected image U as a differentiable function of the kernel table."""
    return KernelImageFn.apply(table, plan, u, v, w, vis, weight)
