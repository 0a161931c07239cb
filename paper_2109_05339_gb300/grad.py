"""Differentiation pattern: the slice loss, its gradient and a gradient-based
merge, with slices recomputed chunk by chunk instead of stored.

loss(x) = 1/2 sum_{i,p} D_p (S_i x - b_ip)^2 + lambda/2 |x - x0|^2, with S_i x
the slice of model x at image i's orientation (Sec. II-A) and b = b_scale *
images. Its gradient S^T D (S x - b) + lambda (x - x0) is the type-1 adjoint
of the weighted residual (Sec. II-C). On models even in n (real, Friedel-
symmetric intensities) S^T D S equals Re(A^H D A), so minimising this loss is
the Tikhonov problem of Eq. 2 that CG solves with the Toeplitz operator.

The library computes the residuals, the FP64 loss, the gradient, the normal
operator and the line-searched step (spf_slice_loss_grad,
spf_slice_normal_apply, spf_gradient_step); this module allocates the
workspace and marshals. Each chunk's slices live only in a chunk-sized
workspace while that chunk's residual is formed.

``use_autograd=True`` instead forms the same loss in PyTorch around
SliceModel, whose backward is the library's type-1 adjoint: the user-facing
autograd form of the same gradient.
"""
from __future__ import annotations

import torch

from ._lib import check, lib
from .api import Plan, SliceModel, _f32, _ptr, _stream


def _chunk(plan: Plan, n, P2, chunk):
    c = min(chunk, max(n, 1), plan.max_points // P2) if plan.max_points else min(chunk, max(n, 1))
    if c < 1:
        raise ValueError(f"the plan's max_points ({plan.max_points}) holds no image of {P2} pixels")
    return c


def _check(plan, x, quats, q_lab, images, D):
    d = plan.device
    plan._grid(x, "x")
    _f32(quats, "quats", d)
    _f32(q_lab, "q_lab", d)
    _f32(images, "images", d, (quats.shape[0], q_lab.shape[0]))
    if D is not None:
        _f32(D, "D", d, (q_lab.shape[0],))


def loss_and_grad(plan: Plan, x, quats, q_lab, images, b_scale, lam=0.0, x0=None, D=None,
                  chunk=4096, use_autograd=False):
    """(loss as a float64 device scalar, gradient) accumulated over image chunks."""
    n, P2 = quats.shape[0], q_lab.shape[0]
    if use_autograd:
        grad = torch.zeros_like(x)
        loss = torch.zeros((), dtype=torch.float64, device=x.device)
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            xr = x.detach().requires_grad_(True)
            s = SliceModel.apply(xr, quats[c0:c1], q_lab, plan)
            r = s - images[c0:c1] * b_scale
            w = r if D is None else r * D
            part = 0.5 * (r * w).sum(dtype=torch.float64)
            part.backward()
            grad += xr.grad
            loss += part.detach()
        if lam and x0 is not None:
            dx = x - x0
            loss += 0.5 * lam * (dx * dx).sum(dtype=torch.float64)
            grad += lam * dx
        return loss, grad
    _check(plan, x, quats, q_lab, images, D)
    c = _chunk(plan, n, P2, chunk)
    work = torch.empty(c * P2, dtype=torch.float32, device=x.device)
    grad = torch.empty_like(x)
    loss = torch.zeros(1, dtype=torch.float64, device=x.device)
    check(lib.spf_slice_loss_grad(plan._h, _ptr(x), _ptr(x0 if lam else None), _ptr(quats), n, _ptr(q_lab), P2,
                                  _ptr(images), float(b_scale), _ptr(D), float(lam), c, _ptr(work), _ptr(loss),
                                  _ptr(grad), _stream(plan.device)))
    return loss[0], grad


def hessian_apply(plan: Plan, v, quats, q_lab, lam=0.0, D=None, chunk=4096):
    """S^T D S v + lambda v, by one slice and one adjoint per chunk."""
    n, P2 = quats.shape[0], q_lab.shape[0]
    c = _chunk(plan, n, P2, chunk)
    work = torch.empty(c * P2, dtype=torch.float32, device=v.device)
    out = torch.empty_like(v)
    check(lib.spf_slice_normal_apply(plan._h, _ptr(v), _ptr(quats), n, _ptr(q_lab), P2, _ptr(D), float(lam), c,
                                     _ptr(work), _ptr(out), _stream(plan.device)))
    return out


def gradient_merge(plan: Plan, x0, quats, q_lab, images, b_scale, lam, iters, D=None,
                   chunk=4096):
    """Steepest descent with exact line search on the quadratic loss, every
    step on the device (spf_gradient_step). Returns the iterate and the loss
    history (iters + 1 values, read back once at the end)."""
    n, P2 = quats.shape[0], q_lab.shape[0]
    _check(plan, x0, quats, q_lab, images, D)
    c = _chunk(plan, n, P2, chunk)
    x = x0.clone()
    work = torch.empty(c * P2, dtype=torch.float32, device=x0.device)
    g = torch.empty_like(x0)
    Hg = torch.empty_like(x0)
    hist = torch.zeros(iters + 1, dtype=torch.float64, device=x0.device)
    s = _stream(plan.device)
    for k in range(iters):
        check(lib.spf_gradient_step(plan._h, _ptr(x), _ptr(x0), _ptr(quats), n, _ptr(q_lab), P2, _ptr(images),
                                    float(b_scale), _ptr(D), float(lam), c, _ptr(work), _ptr(g), _ptr(Hg),
                                    _ptr(hist[k:k + 1]), s))
    check(lib.spf_slice_loss_grad(plan._h, _ptr(x), _ptr(x0), _ptr(quats), n, _ptr(q_lab), P2, _ptr(images),
                                  float(b_scale), _ptr(D), float(lam), c, _ptr(work), _ptr(hist[iters:]), _ptr(g), s))
    return x, [float(v) for v in hist.cpu()]
