"""Parity at the full c2 size (81^3 model, 128x128 detector, 10^4 orientations,
10^4 images) in the launch configuration bench.py times: one slicing call for
all orientations, one merge call for all images, one match over 10^4 x 10^4.
The oracle checks sampled outputs one by one (direct sums in FP64) and
properties that hold at any size."""
import numpy as np
import pytest

import synth
from oracle import matching, nudft
from oracle.rotation import nufft_points
from tests.gpu_util import f32, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    import torch
    from paper_2109_05339_gb300 import Plan
    pb = synth.make_problem("c2")
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    M = pb.quats.shape[0]
    plan = Plan(N, 1.0, 1e-6, max_points=M * P2)
    d = dict(pb=pb, plan=plan, N=N, P2=P2, M=M,
             A=to_dev(pb.A.astype(np.float32)), quats=to_dev(pb.quats.astype(np.float32)),
             qlab=to_dev(pb.q_lab.astype(np.float32)))
    yield d
    plan.close()
    torch.cuda.empty_cache()


def test_slicing_sampled_outputs(c2):
    pb, plan = c2["pb"], c2["plan"]
    s = plan.slice_model(c2["A"], c2["quats"], c2["qlab"])
    plan.status()
    rng = np.random.default_rng(21)
    j = rng.integers(0, c2["M"], 256)
    p = rng.integers(0, c2["P2"], 256)
    got = s[j, p].cpu().numpy().astype(np.float64)
    q32 = f32(pb.quats.astype(np.float32))
    l32 = f32(pb.q_lab.astype(np.float32))
    t = np.stack([nufft_points(q32[j[k]:j[k] + 1], l32[p[k]:p[k] + 1], c2["N"], 1.0)[0, 0]
                  for k in range(256)])
    ref = nudft.type2(f32(pb.A.astype(np.float32)), t).real
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err


def test_point_set_slicing_sampled_outputs(c2):
    """The slicing the M-TIP driver runs (orientation set sorted once, the
    tensor-core interpolation) at the full size: sampled outputs against the
    FP64 direct sum, and the whole slice stack against the per-call path."""
    from paper_2109_05339_gb300 import PointSet
    pb, plan = c2["pb"], c2["plan"]
    ps = PointSet(plan, c2["quats"], c2["qlab"])
    s = ps.slice(c2["A"])
    plan.status()
    rng = np.random.default_rng(23)
    j = rng.integers(0, c2["M"], 256)
    p = rng.integers(0, c2["P2"], 256)
    got = s[j, p].cpu().numpy().astype(np.float64)
    q32 = f32(pb.quats.astype(np.float32))
    l32 = f32(pb.q_lab.astype(np.float32))
    t = np.stack([nufft_points(q32[j[k]:j[k] + 1], l32[p[k]:p[k] + 1], c2["N"], 1.0)[0, 0]
                  for k in range(256)])
    ref = nudft.type2(f32(pb.A.astype(np.float32)), t).real
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err
    whole = plan.slice_model(c2["A"], c2["quats"], c2["qlab"])
    d = float((s.double() - whole.double()).norm() / whole.double().norm())
    assert d < 2e-6, d
    ps.close()


def test_merge_sampled_modes_and_kernel(c2):
    import torch
    pb, plan, N, P2 = c2["pb"], c2["plan"], c2["N"], c2["P2"]
    rng = np.random.default_rng(22)
    n_img = pb.img_quats.shape[0]
    images = rng.poisson(0.06, (n_img, P2)).astype(np.float32)
    iq = to_dev(pb.img_quats.astype(np.float32))
    rhs, khat = plan.merge_images(to_dev(images), iq, c2["qlab"], b_scale=0.5)
    plan.status()
    rhs = rhs.cpu().numpy().astype(np.float64)
    # Toeplitz kernel K(d) back from its spectrum (FP64 inverse FFT on the host)
    PT = plan.PT
    K = np.fft.ifftn(khat.cpu().numpy().astype(np.float64)).real
    modes = np.array([[0, 0, 0], [3, -2, 1], [-40, 17, 40], [11, 0, -29]], dtype=np.float64)
    dmodes = np.array([[0, 0, 0], [5, -9, 2], [-80, 33, 80], [70, -1, -45]], dtype=np.float64)
    q32 = f32(pb.img_quats.astype(np.float32))
    l32 = f32(pb.q_lab.astype(np.float32))
    v = f32(images).reshape(-1) * 0.5
    acc_r = np.zeros(len(modes))
    acc_k = np.zeros(len(dmodes))
    for c0 in range(0, n_img, 250):
        t = nufft_points(q32[c0:c0 + 250], l32, N, 1.0).reshape(-1, 3)
        acc_r += np.cos(t @ modes.T).T @ v[c0 * P2:(c0 + 250) * P2]
        acc_k += np.cos(t @ dmodes.T).sum(axis=0)
    Mh = (N - 1) // 2
    got_r = np.array([rhs[int(z) + Mh, int(y) + Mh, int(x) + Mh] for x, y, z in modes])
    got_k = np.array([K[int(z) % PT, int(y) % PT, int(x) % PT] for x, y, z in dmodes])
    scale_r = np.abs(v).sum()
    scale_k = float(n_img * P2)
    assert np.all(np.abs(got_r - acc_r) < 1e-5 * scale_r), (got_r, acc_r)
    assert np.all(np.abs(got_k - acc_k) < 1e-5 * scale_k), (got_k, acc_k)
    torch.cuda.synchronize()


def test_toeplitz_equals_direct_operator_and_cg_residual(c2):
    import torch
    pb, plan, N, P2 = c2["pb"], c2["plan"], c2["N"], c2["P2"]
    iq = to_dev(pb.img_quats.astype(np.float32))
    _, khat = plan.merge_images(None, iq, c2["qlab"], want_rhs=False)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(23)
    x = torch.randn((N,) * 3, device="cuda", generator=gen)
    x = 0.5 * (x + x.flip(0, 1, 2))              # even: Re A^H A x = S^T S x
    lam = 1e-3 * iq.shape[0] * P2
    hx = plan.toeplitz_apply(khat, lam, x)
    sx = plan.slice_model(x, iq, c2["qlab"])
    direct = plan.slice_adjoint(sx, iq, c2["qlab"]) + lam * x
    err = float((hx - direct).double().norm() / direct.double().norm())
    assert err < 1e-5, err
    # CG: the recursive residual equals b~ - H x recomputed with the operator
    rhs = plan.slice_adjoint(sx, iq, c2["qlab"])            # data consistent with x
    x0 = torch.zeros_like(x)
    hist = torch.zeros(11, dtype=torch.float64, device="cuda")
    xk = plan.cg_solve(khat, lam, rhs, x0, 10, res_hist=hist)
    r = rhs + lam * x0 - plan.toeplitz_apply(khat, lam, xk)
    h = hist.cpu().numpy()
    assert abs(float(r.double().norm()) - h[-1]) < 1e-3 * h[0]
    assert h[-1] < h[0]


def test_matching_10k_by_10k_sampled_images():
    import torch
    from paper_2109_05339_gb300 import Matcher
    rng = np.random.default_rng(24)
    M = n_img = 10_000
    P = 128
    Y = synth.smooth_rows(rng, M, P)
    pick = rng.integers(0, M, n_img)
    X = synth.poisson_counts(rng, 0.5 * Y[pick])          # counts at scale 0.5
    scale = np.float32(2.0)
    m = Matcher(n_img, M, P * P, "bf16", 8)
    Xd, Yd = to_dev(X), to_dev(Y)
    m.set_images(Xd, float(scale))
    m.add_slices(Yd)
    r = m.results()
    m.status()
    best = r["best"].cpu().numpy()
    d1 = r["d1"].cpu().numpy()
    sample = rng.choice(n_img, 64, replace=False)
    Xs = f32(X[sample]) * float(scale)
    ref = matching.match(Xs, f32(Y), d=matching.distances_expanded(Xs, f32(Y)))
    ok = ref["margin"] > 1e-4
    assert ok.sum() >= 32
    np.testing.assert_array_equal(best[sample][ok], ref["best"][ok])
    np.testing.assert_allclose(d1[sample][ok], ref["d1"][ok], rtol=1e-4)
    m.close()
    torch.cuda.empty_cache()
