"""Every built kernel width: tolerances eps = 1e-4 .. 1e-7 select w = 5 .. 8
(w = ceil(log10(1/eps)) + 1). For each, point-set slicing (tensor-core
interpolation) and the class-sum merge (register-run spreading: paired-cell
windows for w < 8, single-cell windows for w = 8) against the FP64 oracle,
with the tolerance scaled to eps."""
import numpy as np
import pytest

from oracle import merge, nufft, rotation
from tests.gpu_util import f32, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps,w", [(1e-4, 5), (1e-5, 6), (1e-6, 7), (1e-7, 8)])
def test_slice_and_merge_every_width(eps, w):
    import torch
    from paper_2109_05339_gb300 import Plan, PointSet
    pb = problem("c1")
    N, P2, M = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0]
    plan = Plan(N, 1.0, eps, max_points=M * P2)
    assert plan.w == w
    quats = to_dev(pb.quats.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    ps = PointSet(plan, quats, qlab)
    A = to_dev(pb.A.astype(np.float32))
    sl = ps.slice(A)
    plan.status()
    t = rotation.nufft_points(f32(pb.quats.astype(np.float32)), f32(pb.q_lab.astype(np.float32)),
                              N, 1.0).reshape(-1, 3)
    ref = nufft.type2(f32(pb.A.astype(np.float32)), t).real.reshape(M, P2)
    tol = max(20 * eps, 1e-5)
    assert rel_l2(sl.cpu().numpy(), ref) < tol

    rng = np.random.default_rng(41)
    n_img = 173
    images = rng.poisson(6.0, (n_img, P2)).astype(np.float32)
    best = rng.integers(0, M, n_img).astype(np.int32)
    rhs, khat = ps.merge(to_dev(images), to_dev(best, torch.int32), b_scale=0.5)
    plan.status()
    tb = t.reshape(M, P2, 3)[best].reshape(-1, 3)
    ones = np.ones(tb.shape[0])
    ref_rhs = merge.rhs(f32(images).reshape(-1) * 0.5, tb, ones, N)
    ref_khat = merge.kernel_hat(merge.toeplitz_kernel(tb, ones, N), N)
    assert rel_l2(rhs.cpu().numpy(), ref_rhs) < tol
    assert rel_l2(khat.cpu().numpy(), ref_khat) < tol
    ps.close()
    plan.close()
