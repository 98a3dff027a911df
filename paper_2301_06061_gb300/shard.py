"""Multi-GPU imaging by w-plane sharding: each process (one GPU) images a range of
w-planes and the partial images are summed by one collective.

The paper distributes the (u, v, w) mesh over MPI tasks as slabs and reduces their
partial results (section 3.1, the slab decomposition; section 3.2, the reduce).  Here
the unit of work is the w-plane: Eq. 2 is a sum over planes and the grid correction is
linear, so partial images of plane ranges that partition the planes add up to the whole
image.  This module holds the host logic only -- the split of the planes and the
reduce -- so that it runs unchanged on gloo (CPU) and NCCL (GPU) process groups; the
imaging itself is ``wst_image_range``.
"""
from __future__ import annotations


def plane_ranges(n_planes: int, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges [b, e) of the global planes, one per rank, as equal as they can
    be (sizes differ by at most one plane; the first ranks take the larger ones).  A
    plane's cost is dominated by its transforms, which do not depend on its visibility
    count, so equal plane counts balance the ranks."""
    if n_planes < 0 or world < 1:
        raise ValueError("n_planes >= 0 and world >= 1 required")
    q, r = divmod(n_planes, world)
    out, b = [], 0
    for k in range(world):
        e = b + q + (1 if k < r else 0)
        out.append((b, e))
        b = e
    return out


def owned(planes, begin: int, end: int):
    """Mask of the visibilities whose global plane (-1 for dropped or non-finite ones,
    which no rank images) lies in [begin, end)."""
    return (planes >= begin) & (planes < end)


def reduce_images(image, dist, group=None) -> None:
    """Sum the ranks' partial images in place on every rank (one all-reduce).  Complex
    tensors are reduced as their real views (NCCL and gloo sum real types)."""
    if dist is None:
        return
    view = image.view(image.real.dtype) if image.is_complex() else image
    dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
