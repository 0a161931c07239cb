"""Differentiation (config 4 shapes): SliceModel's hand-written backward (the
type-1 adjoint) against the FP64 oracle gradient and against central finite
differences; the adjoint identity at the full 50,000-image size; and a
gradient-based merge compared with the Toeplitz CG over 20 iterations."""
import numpy as np
import pytest

import synth
from oracle import slicing
from tests.gpu_util import f32, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c4():
    import torch  # noqa: F401
    pb = synth.make_problem("c4", n_img=6)
    return pb


def test_gradient_matches_oracle(c4):
    import torch
    from paper_2109_05339_gb300 import Plan, SliceModel
    pb = c4
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    quats = pb.img_quats[:3].astype(np.float32)
    qlab = pb.q_lab.astype(np.float32)
    A = pb.A.astype(np.float32)
    rng = np.random.default_rng(41)
    b = rng.poisson(5.0, (3, P2)).astype(np.float32) * np.float32(0.01)
    plan = Plan(N, 1.0, 1e-6, max_points=3 * P2)
    Ad = to_dev(A).requires_grad_(True)
    s = SliceModel.apply(Ad, to_dev(quats), to_dev(qlab), plan)
    loss = 0.5 * ((s.double() - to_dev(b).double()) ** 2).sum()
    loss.backward()
    g = Ad.grad.cpu().numpy()
    g_ref = slicing.loss_grad(f32(A), f32(quats), f32(qlab), f32(b), 1.0)
    assert rel_l2(g, g_ref) < 1e-4
    plan.status()


def test_loss_and_gradient_match_oracle_on_an_image_subsample():
    """The library's chunked loss and gradient (spf_slice_loss_grad) on 16
    images of 128 x 128 at the c4 size (101^3 model, 262,144 points, three
    chunks with a ragged last one), with beam-stop weights D and the ridge
    term, against the FP64 oracle's slices and adjoint."""
    from paper_2109_05339_gb300 import Plan
    from paper_2109_05339_gb300.grad import loss_and_grad
    pb = synth.make_problem("c4", n_img=16)
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    quats = pb.img_quats.astype(np.float32)
    qlab = pb.q_lab.astype(np.float32)
    A = pb.A.astype(np.float32)
    rng = np.random.default_rng(43)
    b = rng.poisson(4.0, (16, P2)).astype(np.float32)
    D = synth.beamstop_mask(pb.cfg.P, 10.0)
    x0 = (0.9 * A).astype(np.float32)
    scale, lam = np.float32(0.01), 3.0
    plan = Plan(N, 1.0, 1e-6, max_points=6 * P2)
    loss, g = loss_and_grad(plan, to_dev(A), to_dev(quats), to_dev(qlab), to_dev(b), float(scale), lam, to_dev(x0),
                            D=to_dev(D), chunk=6)
    plan.status()
    r = slicing.slice_model(f32(A), f32(quats), f32(qlab), 1.0) - f32(b) * np.float64(scale)
    w = f32(D)[None, :]
    dx = f32(A) - f32(x0)
    ref_loss = 0.5 * float(np.sum(w * r * r)) + 0.5 * lam * float(np.sum(dx * dx))
    ref_g = slicing.slice_adjoint(w * r, f32(quats), f32(qlab), N, 1.0) + lam * dx
    assert abs(float(loss) - ref_loss) < 1e-5 * ref_loss, (float(loss), ref_loss)
    assert rel_l2(g.cpu().numpy(), ref_g) < 1e-4, rel_l2(g.cpu().numpy(), ref_g)
    plan.close()


def test_central_differences_on_64_voxels(c4):
    """The loss is quadratic in A, so central differences equal the gradient
    up to rounding; evaluated with the GPU forward, checked against the GPU
    backward."""
    import torch
    from paper_2109_05339_gb300 import Plan
    from paper_2109_05339_gb300.grad import loss_and_grad
    pb = c4
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    quats = to_dev(pb.img_quats[:4].astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    A = to_dev(pb.A.astype(np.float32))
    rng = np.random.default_rng(42)
    images = to_dev(rng.poisson(3.0, (4, P2)).astype(np.float32))
    scale = 0.02
    plan = Plan(N, 1.0, 1e-6, max_points=4 * P2)
    _, g = loss_and_grad(plan, A, quats, qlab, images, scale)
    g = g.cpu().numpy().astype(np.float64)
    gmax = np.abs(g).max()
    vox = rng.integers(0, N, (64, 3))
    h = 0.05 * float(A.abs().max())
    for z, y, x in vox:
        e = torch.zeros_like(A)
        e[z, y, x] = h
        lp, _ = loss_and_grad(plan, A + e, quats, qlab, images, scale)
        lm, _ = loss_and_grad(plan, A - e, quats, qlab, images, scale)
        fd = (float(lp) - float(lm)) / (2 * h)
        assert abs(fd - g[z, y, x]) < 2e-3 * gmax, (z, y, x, fd, g[z, y, x])


def test_adjoint_identity_at_full_c4_size():
    """<S x, r> = <x, S^T r> over 50,000 images of 128x128 (8.2e8 points),
    in the launch configuration of the chunked merge."""
    import torch
    from paper_2109_05339_gb300 import Plan
    pb = synth.make_problem("c4")
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    chunk = 10_000
    plan = Plan(N, 1.0, 1e-6, max_points=chunk * P2)
    quats = to_dev(pb.img_quats.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    x = torch.randn((N,) * 3, device="cuda", generator=gen)
    x = 0.5 * (x + x.flip(0, 1, 2))
    lhs = 0.0
    sx2 = 0.0
    r2 = 0.0
    back = torch.zeros_like(x)
    for c0 in range(0, quats.shape[0], chunk):
        q = quats[c0:c0 + chunk]
        r = torch.randn((q.shape[0], P2), device="cuda", generator=gen)
        sx = plan.slice_model(x, q, qlab)
        lhs += float((sx.double() * r.double()).sum())
        sx2 += float((sx.double() ** 2).sum())
        r2 += float((r.double() ** 2).sum())
        plan.slice_adjoint(r, q, qlab, out=back, accumulate=c0 > 0)
    rhs = float((x.double() * back.double()).sum())
    assert abs(lhs - rhs) < 1e-5 * np.sqrt(sx2 * r2)
    plan.status()


def test_gradient_merge_versus_cg():
    """Steepest descent with exact line search on the Tikhonov loss (slices
    recomputed per chunk) and CG on the Toeplitz form minimise the same
    quadratic; after 20 iterations CG's loss is no higher, and both are far
    below the starting loss."""
    import torch
    from paper_2109_05339_gb300 import Plan
    from paper_2109_05339_gb300.grad import gradient_merge, loss_and_grad
    pb = synth.make_problem("c4", n_img=200)
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    quats = to_dev(pb.img_quats.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    x0 = to_dev(pb.A.astype(np.float32))
    plan = Plan(N, 1.0, 1e-6, max_points=200 * P2)
    clean = plan.slice_model(x0, quats, qlab)
    s = 1e3 / float(clean.double().sum(1).mean())
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    images = torch.poisson(clean * s, generator=gen)
    lam = 1e-3 * 200 * P2
    xg, hist = gradient_merge(plan, x0 * 0.5, quats, qlab, images, 1.0 / s, lam, 20, chunk=100)
    rhs, khat = plan.merge_images(images, quats, qlab, b_scale=1.0 / s)
    # CG solves H x = rhs + lam x0 with x0 the same prior point as the loss
    x0p = x0 * 0.5
    xc = plan.cg_solve(khat, lam, rhs, x0p, 20)
    lg, _ = loss_and_grad(plan, xg, quats, qlab, images, 1.0 / s, lam, x0p, chunk=100)
    lc, _ = loss_and_grad(plan, xc, quats, qlab, images, 1.0 / s, lam, x0p, chunk=100)
    l0 = hist[0]
    assert float(lc) <= float(lg) * (1 + 1e-5)
    assert float(lg) < l0 and float(lc) < l0
    assert all(hist[k + 1] <= hist[k] * (1 + 1e-7) for k in range(len(hist) - 1))
