"""GPU merge (Sec. II-C, Eq. 2): type-1 right-hand side, Toeplitz kernel,
Toeplitz operator and CG against the FP64 oracle."""
import numpy as np
import pytest

from oracle import merge, rotation
from tests.gpu_util import f32, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1_merge():
    import torch
    from paper_2109_05339_gb300 import Plan
    pb = problem("c1")
    N = pb.cfg.N
    rng = np.random.default_rng(77)
    n_img = 100
    quats = pb.quats.astype(np.float32)
    best = pb.img_pick.astype(np.int32)
    images = rng.poisson(30.0, (n_img, pb.q_lab.shape[0])).astype(np.float32)
    qlab = pb.q_lab.astype(np.float32)
    D = (rng.uniform(size=qlab.shape[0]) > 0.05).astype(np.float32)
    b_scale = np.float32(1e-3)
    plan = Plan(N, 1.0, 1e-6, max_points=n_img * qlab.shape[0])
    rhs, khat = plan.merge_images(to_dev(images), to_dev(quats), to_dev(qlab), D=to_dev(D),
                                  b_scale=float(b_scale), orient_idx=to_dev(best, torch.int32))
    t = rotation.nufft_points(f32(quats)[best], f32(qlab), N, 1.0).reshape(-1, 3)
    Dall = np.tile(f32(D), n_img)
    b = f32(images).reshape(-1) * np.float64(b_scale)
    ref_rhs = merge.rhs(b, t, Dall, N)
    K = merge.toeplitz_kernel(t, Dall, N)
    ref_khat = merge.kernel_hat(K, N)
    return dict(plan=plan, rhs=rhs, khat=khat, ref_rhs=ref_rhs, ref_khat=ref_khat, t=t, Dall=Dall,
                N=N, images=images, quats=quats, best=best, qlab=qlab, D=D, b_scale=b_scale)


def test_rhs_and_kernel(c1_merge):
    c = c1_merge
    assert rel_l2(c["rhs"].cpu().numpy(), c["ref_rhs"]) < 1e-5
    assert rel_l2(c["khat"].cpu().numpy(), c["ref_khat"]) < 1e-5
    c["plan"].status()


def test_chunks_accumulate_to_whole(c1_merge):
    import torch
    c = c1_merge
    plan = c["plan"]
    rhs = torch.zeros_like(c["rhs"])
    kh = torch.zeros_like(c["khat"])
    for c0, c1 in [(0, 33), (33, 34), (34, 100)]:
        plan.merge_images(to_dev(c["images"][c0:c1]), to_dev(c["quats"]), to_dev(c["qlab"]),
                          D=to_dev(c["D"]), b_scale=float(c["b_scale"]), rhs=rhs, kernel_hat=kh,
                          accumulate=c0 > 0, orient_idx=to_dev(c["best"][c0:c1], torch.int32))
    assert rel_l2(rhs.cpu().numpy(), c["rhs"].cpu().numpy()) < 1e-6
    assert rel_l2(kh.cpu().numpy(), c["khat"].cpu().numpy()) < 1e-6


def test_deferred_merge_over_chunks_equals_one_call(c1_merge):
    """Chunks spread onto one open merge and transformed once give the
    single-call merge of all images; calls that would overwrite the fine
    grids are refused while the merge is open."""
    import torch
    from paper_2109_05339_gb300 import SpfError
    c = c1_merge
    plan = c["plan"]
    plan.merge_begin()
    for c0, c1 in [(0, 33), (33, 34), (34, 100)]:
        plan.merge_images_add(to_dev(c["images"][c0:c1]), to_dev(c["quats"]), to_dev(c["qlab"]), D=to_dev(c["D"]),
                              b_scale=float(c["b_scale"]), orient_idx=to_dev(c["best"][c0:c1], torch.int32))
    with pytest.raises(SpfError, match="deferred merge is open"):
        plan.slice_model(to_dev(np.zeros((c["N"],) * 3, np.float32)), to_dev(c["quats"]), to_dev(c["qlab"]))
    rhs = torch.empty_like(c["rhs"])
    kh = torch.empty_like(c["khat"])
    plan.merge_finish(rhs, kh)
    plan.status()
    assert rel_l2(rhs.cpu().numpy(), c["rhs"].cpu().numpy()) < 1e-6
    assert rel_l2(kh.cpu().numpy(), c["khat"].cpu().numpy()) < 1e-6
    with pytest.raises(SpfError, match="no deferred merge"):
        plan.merge_finish(rhs, kh)


def test_toeplitz_operator(c1_merge):
    c = c1_merge
    N = c["N"]
    rng = np.random.default_rng(8)
    x = rng.standard_normal((N, N, N)).astype(np.float32)
    lam = 0.7 * float(c["Dall"].sum()) * 1e-3
    y = c["plan"].toeplitz_apply(c["khat"], lam, to_dev(x)).cpu().numpy()
    ref = merge.apply_toeplitz(f32(x), c["ref_khat"], N, lam)
    assert rel_l2(y, ref) < 1e-5
    # and equals the direct operator Re(type1(D type2 x)) + lam x (oracle, Sec. III-A)
    ref_direct = merge.apply_direct(f32(x), c["t"], c["Dall"], lam)
    assert rel_l2(y, ref_direct) < 1e-5


@pytest.mark.parametrize("iters", [1, 5])
def test_cg_matches_oracle(c1_merge, iters):
    import torch
    c = c1_merge
    N = c["N"]
    plan = c["plan"]
    lam = 1e-3 * float(c["Dall"].sum())
    rng = np.random.default_rng(10)
    x0 = (rng.standard_normal((N, N, N)) * 0.01).astype(np.float32)
    hist = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    x = plan.cg_solve(c["khat"], lam, c["rhs"], to_dev(x0), iters, res_hist=hist).cpu().numpy()
    bt = c["ref_rhs"] + lam * f32(x0)
    xr, hr = merge.cg(lambda v: merge.apply_toeplitz(v, c["ref_khat"], N, lam), bt, f32(x0), iters)
    assert rel_l2(x, xr) < 1e-4
    np.testing.assert_allclose(hist.cpu().numpy(), hr, rtol=1e-4)


def test_toeplitz_and_cg_at_generic_fft_sides():
    """N = 21: fine grid 48, Toeplitz grid 90, embedding 48 -- no precompiled
    FFT plan, so the generic passes and the unfused convolution run."""
    import torch
    from paper_2109_05339_gb300 import Plan
    N = 21
    pb = problem("c1")
    qlab = pb.q_lab.astype(np.float32)
    rng = np.random.default_rng(91)
    q = rng.standard_normal((40, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1
    quats = q.astype(np.float32)
    plan = Plan(N, 1.0, 1e-6, max_points=quats.shape[0] * qlab.shape[0])
    assert plan.PT == 48
    images = rng.poisson(20.0, (quats.shape[0], qlab.shape[0])).astype(np.float32)
    rhs, khat = plan.merge_images(to_dev(images), to_dev(quats), to_dev(qlab), b_scale=0.01)
    plan.status()
    t = rotation.nufft_points(f32(quats), f32(qlab), N, 1.0).reshape(-1, 3)
    ones = np.ones(t.shape[0])
    ref_rhs = merge.rhs(f32(images).reshape(-1) * 0.01, t, ones, N)
    ref_khat = merge.kernel_hat(merge.toeplitz_kernel(t, ones, N), N)
    assert rel_l2(rhs.cpu().numpy(), ref_rhs) < 1e-5
    assert rel_l2(khat.cpu().numpy(), ref_khat) < 1e-5
    lam = 1e-3 * float(ones.sum())
    x0 = (rng.standard_normal((N, N, N)) * 0.01).astype(np.float32)
    y = plan.toeplitz_apply(khat, lam, to_dev(x0)).cpu().numpy()
    assert rel_l2(y, merge.apply_toeplitz(f32(x0), ref_khat, N, lam)) < 1e-5
    hist = torch.zeros(4, dtype=torch.float64, device="cuda")
    x = plan.cg_solve(khat, lam, rhs, to_dev(x0), 3, res_hist=hist).cpu().numpy()
    xr, hr = merge.cg(lambda v: merge.apply_toeplitz(v, ref_khat, N, lam), ref_rhs + lam * f32(x0), f32(x0), 3)
    assert rel_l2(x, xr) < 1e-4
    plan.close()


@pytest.mark.parametrize("N,PT", [(35, 72), (101, 216)])
def test_real_input_toeplitz_apply_and_cg(N, PT):
    """Precompiled cube sides: the right-hand side and the kernel spectrum
    (real-input type-1 transforms) against the oracle's merge; the Toeplitz
    apply -- real-input row transforms (two rows per complex line),
    half-spectrum y and z passes with the kernel product inside the z pass,
    and the inverse row transforms -- against the oracle's complex
    convolution with the oracle's kernel; three CG steps on the oracle's
    right-hand side and kernel against the oracle's CG."""
    import torch
    from paper_2109_05339_gb300 import Plan
    pb = problem("c1")
    qlab = pb.q_lab.astype(np.float32)
    rng = np.random.default_rng(N)
    q = rng.standard_normal((40, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1
    quats = q.astype(np.float32)
    plan = Plan(N, 1.0, 1e-6, max_points=quats.shape[0] * qlab.shape[0])
    assert plan.PT == PT
    images = rng.poisson(20.0, (quats.shape[0], qlab.shape[0])).astype(np.float32)
    rhs, khat = plan.merge_images(to_dev(images), to_dev(quats), to_dev(qlab), b_scale=0.01)
    plan.status()
    t = rotation.nufft_points(f32(quats), f32(qlab), N, 1.0).reshape(-1, 3)
    ones = np.ones(t.shape[0])
    ref_rhs = merge.rhs(f32(images).reshape(-1) * 0.01, t, ones, N)
    ref_khat = merge.kernel_hat(merge.toeplitz_kernel(t, ones, N), N)
    assert rel_l2(rhs.cpu().numpy(), ref_rhs) < 1e-5
    assert rel_l2(khat.cpu().numpy(), ref_khat) < 1e-5
    lam = 1e-3 * float(images.size)
    x0 = (rng.standard_normal((N, N, N)) * 0.01).astype(np.float32)
    kh32 = f32(ref_khat.astype(np.float32))
    y = plan.toeplitz_apply(to_dev(kh32), lam, to_dev(x0)).cpu().numpy()
    assert rel_l2(y, merge.apply_toeplitz(f32(x0), kh32, N, lam)) < 1e-5
    hist = torch.zeros(4, dtype=torch.float64, device="cuda")
    rhs32 = f32(ref_rhs.astype(np.float32))
    x = plan.cg_solve(to_dev(kh32), lam, to_dev(rhs32), to_dev(x0), 3, res_hist=hist).cpu().numpy()
    xr, hr = merge.cg(lambda v: merge.apply_toeplitz(v, kh32, N, lam), rhs32 + lam * f32(x0), f32(x0), 3)
    assert rel_l2(x, xr) < 1e-4
    np.testing.assert_allclose(hist.cpu().numpy(), hr, rtol=1e-4)
    plan.close()
