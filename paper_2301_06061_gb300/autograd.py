"""torch.autograd bindings of the imager and of its tabulated kernel.

``ImageFn``: D = A V, forward ``wst_image``, backward ``wst_degrid``.  A is C-linear
in the visibilities, so the vector-Jacobian product torch asks for is the adjoint
A^H applied to the incoming gradient (degridding; the paper's conclusions list it
as the next step).  Both directions run in libwst's CUDA kernels.

``KernelImageFn``: U(table), the image without grid correction as a function of a
tabulated kernel's samples; backward ``wst_kernel_grad``.  The grid correction,
which also depends on the table, is left to differentiable torch code
(``learned.correction_matrix``).

A plan holds one binding of visibilities (and kernel table) at a time, while the
backward pass needs the binding of its own forward pass.  Each forward pass therefore
keeps its inputs and the plan's ``generation``; if the plan has been rebound since
(another forward pass on the same plan, for instance), backward binds them again
before it runs, so every backward pass differentiates its own forward pass.
"""
from __future__ import annotations

import torch

from . import wst


class ImageFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vis, plan, u, v, w, weight, flags):
        vis64 = vis.detach().to(torch.complex64).contiguous()
        plan.set_vis(u, v, w, vis64, weight)
        out = plan.image(flags=flags)
        ctx.plan = plan
        ctx.flags = flags
        ctx.in_dtype = vis.dtype
        ctx.generation = plan.generation
        ctx.save_for_backward(u, v, w, vis64, weight)
        return out if vis.dtype == torch.complex64 else out.to(vis.dtype)

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        u, v, w, vis64, weight = ctx.saved_tensors
        if plan.generation != ctx.generation:  # the plan was rebound after this forward
            plan.set_vis(u, v, w, vis64, weight)
            ctx.generation = plan.generation
        g = grad.detach().to(torch.complex64).contiguous()
        dvis = plan.degrid(g, flags=ctx.flags)
        return dvis.to(ctx.in_dtype), None, None, None, None, None, None


def image(vis, plan, u, v, w, weight=None, flags: int = 0):
    """Differentiable w-stacking image of ``vis`` (complex) on a ``wst.Plan``."""
    return ImageFn.apply(vis, plan, u, v, w, weight, flags)


class KernelImageFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, table, plan, u, v, w, vis, weight):
        tab32 = table.detach().to(torch.float32).contiguous()
        plan.set_kernel_table(tab32)
        plan.set_vis(u, v, w, vis, weight)
        out = plan.image(flags=wst.WST_NO_CORRECTION)
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.save_for_backward(tab32, u, v, w, vis, weight)
        return out

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        tab32, u, v, w, vis, weight = ctx.saved_tensors
        if plan.generation != ctx.generation:  # the plan was rebound after this forward
            plan.set_kernel_table(tab32)
            plan.set_vis(u, v, w, vis, weight)
            ctx.generation = plan.generation
        dtab = plan.kernel_grad(grad.detach().to(torch.complex64).contiguous())
        return dtab, None, None, None, None, None, None


def kernel_image(table, plan, u, v, w, vis, weight=None):
    """Uncorrected image U as a differentiable function of the kernel table."""
    return KernelImageFn.apply(table, plan, u, v, w, vis, weight)
