"""Image-sharded M-TIP over several processes, one GPU each.

Matching is independent per image, and the merge's type-1 sums are linear in
the images: each node sums its own images and the node sums are added
(Sec. II-C). So every rank slices, matches and merges its own images, the
right-hand side A^H D b and the Toeplitz kernel K^ are summed over the ranks,
and every rank then runs the same CG solve on identical inputs. lambda is
scaled by the global image count.

The reduction helpers sit apart from the driver binding (mtip.py) because they
import without the native library: the two-process gloo test runs them on CPU
ranks, and the driver calls them between its merge and solve entry points.
"""
from __future__ import annotations

import torch


def allreduce_sum_(tensors, group=None):
    """Sum each tensor over the ranks of `group`, in place (the collective
    runs on the backend's stream, ordered after the current stream)."""
    import torch.distributed as dist
    for t in tensors:
        if not t.is_contiguous():
            raise ValueError("allreduce_sum_ needs contiguous tensors (it reduces in place)")
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def global_count(n, device, group=None):
    """Sum of the ranks' local counts n (a host value; one small collective)."""
    t = torch.tensor([int(n)], dtype=torch.int64, device=device)
    allreduce_sum_([t], group)
    return int(t.item())
