"""L-curve lambda selection (Sec. II-C) on the GPU against the FP64 oracle:
same lambda grid and CG steps give the same residual / penalty norms and the
same corner; the beam-stop mask enters the merge through D."""
import numpy as np
import pytest

import synth
from oracle import lcurve as olc
from oracle import rotation
from tests.gpu_util import f32, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def test_lcurve_sweep_matches_oracle():
    import torch
    from paper_2109_05339_gb300 import Plan
    from paper_2109_05339_gb300.lcurve import sweep, weighted_sumsq
    pb = problem("c1")
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    rng = np.random.default_rng(81)
    n = 60
    best = rng.integers(0, pb.quats.shape[0], n)
    images = rng.poisson(40.0, (n, P2)).astype(np.float32)
    D = synth.beamstop_mask(pb.cfg.P, 2.5)
    scale = np.float32(1e-2)
    plan = Plan(N, 1.0, 1e-6, max_points=n * P2)
    quats = to_dev(pb.quats.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    Dd = to_dev(D)
    img = to_dev(images)
    rhs, khat = plan.merge_images(img, quats, qlab, D=Dd, b_scale=float(scale),
                                  orient_idx=to_dev(best.astype(np.int32), torch.int32))
    b2 = weighted_sumsq(plan, img, Dd, float(scale))
    x0 = to_dev(pb.A.astype(np.float32))
    lams = np.logspace(-4, 1, 9) * float(D.sum() * n)
    iters = 6
    got = sweep(plan, khat, rhs, x0, lams, iters, b2)
    t = rotation.nufft_points(f32(pb.quats.astype(np.float32))[best],
                              f32(pb.q_lab.astype(np.float32)), N, 1.0).reshape(-1, 3)
    Dall = np.tile(f32(D), n)
    b = f32(images).reshape(-1) * np.float64(scale)
    _, res2, reg2, idx = olc.sweep(t, Dall, b, N, f32(pb.A.astype(np.float32)), lams, iters)
    assert rel_l2(got["res2"], res2) < 1e-4
    assert rel_l2(got["reg2"], reg2) < 5e-3
    assert got["index"] == idx
    plan.status()
