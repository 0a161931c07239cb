"""L-curve choice of the Tikhonov parameter lambda for the merge (Sec. II-C).

For each lambda of a sweep, CG solves Eq. 2 on the device; the library then
computes |A x - b|_D^2 (from the Toeplitz product and the right-hand side, no
pass over the points) and |x - x0|^2 with FP64 reductions. The chosen lambda
maximises the curvature of (log |A x - b|, log |x - x0|) as a function of
log lambda (three-point derivatives on the possibly uneven grid). Only the
few scalars of the curve are read back to the host.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import check, lib
from .api import Plan, _f32, _ptr, _stream


def _deriv(y, s):
    h0 = s[1:-1] - s[:-2]
    h1 = s[2:] - s[1:-1]
    d1 = (-h1 / (h0 * (h0 + h1)) * y[:-2] + (h1 - h0) / (h0 * h1) * y[1:-1]
          + h0 / (h1 * (h0 + h1)) * y[2:])
    d2 = 2.0 * (y[:-2] / (h0 * (h0 + h1)) - y[1:-1] / (h0 * h1) + y[2:] / (h1 * (h0 + h1)))
    return d1, d2


def corner(lams, res2, reg2):
    """Index of the maximum-curvature point of the L-curve (interior points)."""
    s = np.log(np.asarray(lams, dtype=np.float64))
    rho = 0.5 * np.log(np.asarray(res2, dtype=np.float64))
    eta = 0.5 * np.log(np.asarray(reg2, dtype=np.float64))
    r1, r2 = _deriv(rho, s)
    e1, e2 = _deriv(eta, s)
    kappa = (r1 * e2 - r2 * e1) / (r1 * r1 + e1 * e1) ** 1.5
    return int(np.argmax(kappa)) + 1, kappa


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
    """CG solve for every lambda; returns dict(lams, res2, reg2, index, x)."""
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
