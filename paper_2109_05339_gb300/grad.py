"""Differentiation pattern: the slice loss, its gradient, and a gradient-based
merge, with slices recomputed chunk by chunk instead of stored.

loss(x) = 1/2 sum_{i,p} D_p (S_i x - b_ip)^2 + lambda/2 |x - x0|^2, with S_i x
the slice of model x at image i's orientation (Sec. II-A) and b = b_scale *
images. Its gradient S^T D (S x - b) + lambda (x - x0) is the type-1 adjoint
of the weighted residual (Sec. II-C). On models even in n (real, Friedel-
symmetric intensities) S^T D S equals Re(A^H D A), so minimising this loss is
the Tikhonov problem of Eq. 2 that CG solves with the Toeplitz operator.

Each chunk's slices live only while that chunk's residual is formed; the
backward never needs them, so memory holds one chunk, not all images.
"""
from __future__ import annotations

import torch

from .api import Plan, SliceModel


def loss_and_grad(plan: Plan, x, quats, q_lab, images, b_scale, lam=0.0, x0=None, D=None,
                  chunk=4096, use_autograd=False):
    """(loss as a float64 tensor, gradient) accumulated over image chunks."""
    n = quats.shape[0]
    grad = torch.zeros_like(x)
    loss = torch.zeros((), dtype=torch.float64, device=x.device)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        q = quats[c0:c1]
        b = images[c0:c1] * b_scale
        if use_autograd:
            xr = x.detach().requires_grad_(True)
            s = SliceModel.apply(xr, q, q_lab, plan)
            r = s - b
            w = r if D is None else r * D
            part = 0.5 * (r * w).sum(dtype=torch.float64)
            part.backward()
            grad += xr.grad
            loss += part.detach()
        else:
            s = plan.slice_model(x, q, q_lab)
            r = s.sub_(b)
            if D is not None:
                loss += 0.5 * (r * r * D).sum(dtype=torch.float64)
                r.mul_(D)
            else:
                loss += 0.5 * (r * r).sum(dtype=torch.float64)
            plan.slice_adjoint(r, q, q_lab, out=grad, accumulate=True)
    if lam and x0 is not None:
        d = x - x0
        loss += 0.5 * lam * (d * d).sum(dtype=torch.float64)
        grad += lam * d
    return loss, grad


def hessian_apply(plan: Plan, v, quats, q_lab, lam=0.0, D=None, chunk=4096):
    """S^T D S v + lambda v, by one slice and one adjoint per chunk."""
    out = torch.zeros_like(v)
    n = quats.shape[0]
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        s = plan.slice_model(v, quats[c0:c1], q_lab)
        if D is not None:
            s.mul_(D)
        plan.slice_adjoint(s, quats[c0:c1], q_lab, out=out, accumulate=True)
    if lam:
        out += lam * v
    return out


def gradient_merge(plan: Plan, x0, quats, q_lab, images, b_scale, lam, iters, D=None,
                   chunk=4096):
    """Steepest descent with exact line search on the quadratic loss.

    Returns the iterate and the loss history (iters + 1 values)."""
    x = x0.clone()
    hist = []
    for _ in range(iters):
        loss, g = loss_and_grad(plan, x, quats, q_lab, images, b_scale, lam, x0, D, chunk)
        hist.append(float(loss))
        Hg = hessian_apply(plan, g, quats, q_lab, lam, D, chunk)
        gg = float((g.double() * g.double()).sum())
        gHg = float((g.double() * Hg.double()).sum())
        if gHg <= 0.0 or gg == 0.0:
            break
        x -= (gg / gHg) * g
    loss, _ = loss_and_grad(plan, x, quats, q_lab, images, b_scale, lam, x0, D, chunk)
    hist.append(float(loss))
    return x, hist
