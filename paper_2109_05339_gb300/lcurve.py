"""L-curve choice of the Tikhonov parameter lambda for the merge (Sec. II-C).

For each lambda of a sweep, CG solves Eq. 2 on the device; the library then
computes |A x - b|_D^2 (from the Toeplitz product and the right-hand side, no
pass over the points) and |x - x0|^2 with FP64 reductions, and picks the
lambda of maximum curvature of (log |A x - b|_D, log |x - x0|) over
log lambda (spf_lcurve_corner). This module only marshals: the few scalars of
the curve are read back and passed to the library's corner search.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import check, lib
from .api import Plan, _f32, _ptr, _stream


def corner(lams, res2, reg2):
    """Index of the maximum-curvature point of the L-curve, and the curvature
    at the interior points (computed by the library)."""
    lams = np.ascontiguousarray(lams, dtype=np.float64)
    res2 = np.ascontiguousarray(res2, dtype=np.float64)
    reg2 = np.ascontiguousarray(reg2, dtype=np.float64)
    n = lams.shape[0]
    kappa = np.zeros(max(n - 2, 0), dtype=np.float64)
    idx = C.c_int()
    check(lib.spf_lcurve_corner(lams.ctypes.data_as(C.c_void_p), res2.ctypes.data_as(C.c_void_p),
                                reg2.ctypes.data_as(C.c_void_p), n, C.byref(idx),
                                kappa.ctypes.data_as(C.c_void_p)))
    return idx.value, kappa


def weighted_sumsq(plan: Plan, images, D=None, scale=1.0, out=None, accumulate=False):
    """b.D b of the scaled images as a device float64 scalar (shape (1,))."""
    d = plan.device
    _f32(images, "images", d)
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=images.device)
    check(lib.spf_weighted_sumsq(plan._h, _ptr(images), images.shape[0], images.shape[1], _ptr(D),
                                 C.c_float(scale), _ptr(out), int(bool(accumulate)), _stream(d)))
    return out


def sweep(plan: Plan, kernel_hat, rhs, x0, lams, iters, b_norm2):
    """CG solve for every lambda; returns dict(lams, res2, reg2, index, kappa, x, xs)."""
    d = plan.device
    vals = torch.zeros((len(lams), 2), dtype=torch.float64, device=x0.device)
    xs = []
    for k, lam in enumerate(lams):
        x = plan.cg_solve(kernel_hat, lam, rhs, x0, iters)
        check(lib.spf_cg_objective(plan._h, _ptr(kernel_hat), _ptr(rhs), _ptr(x), _ptr(x0),
                                   _ptr(b_norm2), _ptr(vals[k]), _stream(d)))
        xs.append(x)
    v = vals.cpu().numpy()
    idx, kappa = corner(lams, v[:, 0], v[:, 1])
    return {"lams": np.asarray(lams), "res2": v[:, 0], "reg2": v[:, 1], "index": idx,
            "kappa": kappa, "x": xs[idx], "xs": xs}
