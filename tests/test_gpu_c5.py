"""Parity at the largest one-GPU size: 151^3 model, 192x192 Ewald detector
(36,864-pixel rows), fine grid 320, Toeplitz fine grid 640, circulant
embedding 320 -- in the launch configuration bench.py times: a point set of
one 10,000-orientation chunk, sliced by the tensor-core interpolation and
merged by class sums; the real-input Toeplitz apply and CG on the 320^3
embedding; BF16 and FP8 matching of 36,864-pixel rows with ragged tiles.

The oracle checks sampled outputs one by one (direct sums in FP64), the
Toeplitz apply and CG against its own FP64 operator and CG on a kernel it
computed itself, and matching against its brute-force distances."""
import numpy as np
import pytest

import synth
from oracle import matching, merge, nudft
from oracle.rotation import quat_to_matrix, radians_per_q
from tests.gpu_util import f32, rel_l2, to_dev

pytestmark = pytest.mark.gpu
CHUNK = 10_000   # orientations per point set, as the bench streams them


@pytest.fixture(scope="module")
def c5():
    import torch
    from paper_2109_05339_gb300 import Plan, PointSet
    pb = synth.make_problem("c5", n_orient=CHUNK, n_img=1)
    N, P2 = pb.cfg.N, pb.q_lab.shape[0]
    plan = Plan(N, 1.0, 1e-6, max_points=CHUNK * P2)
    assert (plan.nf, plan.nfT, plan.PT, P2) == (320, 640, 320, 36864)
    quats = to_dev(pb.quats.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    ps = PointSet(plan, quats, qlab)
    d = dict(pb=pb, plan=plan, ps=ps, N=N, P2=P2, quats=quats, qlab=qlab,
             A=to_dev(pb.A.astype(np.float32)), q32=f32(pb.quats.astype(np.float32)),
             l32=f32(pb.q_lab.astype(np.float32)))
    yield d
    ps.close()
    plan.close()
    torch.cuda.empty_cache()


def _points(c, j, p):
    """FP64 NUFFT coordinates t = 2 pi dr R(quat_j) q_p of the FP32 inputs, per pair."""
    R = quat_to_matrix(c["q32"][j])
    return radians_per_q(c["N"], 1.0) * np.einsum("kab,kb->ka", R, c["l32"][p])


def test_c5_point_set_slicing_sampled_outputs(c5):
    """Slices of the 10,000-orientation point set (3.7e8 points) at sampled
    (orientation, pixel) pairs -- the last orientation and the detector
    corners included -- against the FP64 direct sum; the point-set path
    against the per-call path on a ragged block of orientations."""
    plan, ps = c5["plan"], c5["ps"]
    s = ps.slice(c5["A"])
    plan.status()
    rng = np.random.default_rng(51)
    P2 = c5["P2"]
    j = np.concatenate([rng.integers(0, CHUNK, 120), [CHUNK - 1, CHUNK - 1, 0, 0]])
    p = np.concatenate([rng.integers(0, P2, 120), [0, P2 - 1, 191, P2 - 192]])
    got = s[j, p].cpu().numpy().astype(np.float64)
    ref = nudft.type2(f32(c5["pb"].A.astype(np.float32)), _points(c5, j, p)).real
    err = rel_l2(got, ref)
    assert err < 1e-5, err
    blk = slice(CHUNK - 37, CHUNK)
    whole = plan.slice_model(c5["A"], c5["quats"][blk].contiguous(), c5["qlab"])
    d = rel_l2(s[blk].cpu().numpy(), whole.cpu().numpy())
    assert d < 2e-6, d


def test_c5_merge_sampled_modes_and_kernel(c5):
    """Class-sum merge of 4,000 sparse Poisson images (500 photons over 36,864
    pixels, a beam-stop mask) matched to 200 of the chunk's orientations:
    right-hand-side modes and Toeplitz-kernel offsets (from K^ by an FP64
    inverse FFT on the host) against the FP64 direct sums over every point."""
    import torch
    plan, ps, N, P2 = c5["plan"], c5["ps"], c5["N"], c5["P2"]
    rng = np.random.default_rng(52)
    n_img = 4000
    classes = np.sort(rng.choice(CHUNK, 200, replace=False))
    oidx = classes[rng.integers(0, 200, n_img)].astype(np.int32)
    images = rng.poisson(500.0 / P2, (n_img, P2)).astype(np.float32)
    D = synth.beamstop_mask(192, 8.0)
    b_scale = np.float32(0.25)
    rhs, khat = ps.merge(to_dev(images), to_dev(oidx, torch.int32), D=to_dev(D), b_scale=float(b_scale))
    plan.status()
    rhs = rhs.cpu().numpy().astype(np.float64)
    K = np.fft.ifftn(khat.cpu().numpy().astype(np.float64)).real
    PT, Mh = plan.PT, (N - 1) // 2
    # right-hand side: sum over the nonzero weighted pixels of v cos(n . t)
    i_nz, p_nz = np.nonzero(images * D[None, :])
    v = f32(images[i_nz, p_nz]) * f32(D[p_nz]) * np.float64(b_scale)
    t = _points(c5, oidx[i_nz], p_nz)
    modes = np.array([[0, 0, 0], [3, -2, 1], [-75, 40, 75], [11, 0, -29], [75, 75, -75]], dtype=np.float64)
    ref_r = np.cos(t @ modes.T).T @ v
    got_r = np.array([rhs[int(z) + Mh, int(y) + Mh, int(x) + Mh] for x, y, z in modes])
    assert np.all(np.abs(got_r - ref_r) < 1e-5 * np.abs(v).sum()), (got_r, ref_r)
    # Toeplitz kernel: K(d) = sum_j count_j sum_p D_p cos(d . t_jp)
    dmodes = np.array([[0, 0, 0], [5, -9, 2], [-150, 33, 150], [140, -1, -45]], dtype=np.float64)
    cls, cnt = np.unique(oidx, return_counts=True)
    ref_k = np.zeros(len(dmodes))
    pix = np.arange(P2)
    for c, m in zip(cls, cnt):
        tj = _points(c5, np.full(P2, c), pix)
        ref_k += m * (np.cos(tj @ dmodes.T).T @ f32(D))
    got_k = np.array([K[int(z) % PT, int(y) % PT, int(x) % PT] for x, y, z in dmodes])
    assert np.all(np.abs(got_k - ref_k) < 1e-5 * n_img * float(D.sum())), (got_k, ref_k)


def _even_kernel(N):
    """A real, even kernel on the (2N-1)^3 offsets whose Toeplitz operator is
    positive definite: a sum of two isotropic Gaussians (positive-definite
    functions), stored [d_z][d_y][d_x]."""
    d = np.arange(-(N - 1), N, dtype=np.float64) ** 2
    r2 = d[:, None, None] + d[None, :, None] + d[None, None, :]
    return np.exp(-r2 / 18.0) + 0.3 * np.exp(-r2 / 200.0)


def test_c5_toeplitz_apply_and_cg_against_oracle(c5):
    """The real-input Toeplitz apply (151^3 vector in the 320^3 embedding) and
    three CG steps on a K^ the oracle built (FP32-rounded, as the GPU gets
    it), against the oracle's complex FFT convolution and FP64 CG."""
    import torch
    plan, N = c5["plan"], c5["N"]
    Kh = f32(merge.kernel_hat(_even_kernel(N), N).astype(np.float32))
    kh_d = to_dev(Kh)
    rng = np.random.default_rng(53)
    x = rng.standard_normal((N, N, N)).astype(np.float32)
    lam = 0.05
    y = plan.toeplitz_apply(kh_d, lam, to_dev(x)).cpu().numpy()
    ref = merge.apply_toeplitz(f32(x), Kh, N, lam)
    assert rel_l2(y, ref) < 1e-5, rel_l2(y, ref)
    rhs = rng.standard_normal((N, N, N)).astype(np.float32)
    x0 = (0.1 * rng.standard_normal((N, N, N))).astype(np.float32)
    hist = torch.zeros(4, dtype=torch.float64, device="cuda")
    xg = plan.cg_solve(kh_d, lam, to_dev(rhs), to_dev(x0), 3, res_hist=hist).cpu().numpy()
    xr, hr = merge.cg(lambda v: merge.apply_toeplitz(v, Kh, N, lam), f32(rhs) + lam * f32(x0), f32(x0), 3)
    assert rel_l2(xg, xr) < 1e-4, rel_l2(xg, xr)
    np.testing.assert_allclose(hist.cpu().numpy(), hr, rtol=1e-4)


def test_c5_matching_grid_schedule_many_image_tiles():
    """The CTA-grid tile schedule the matcher picks for the c5 launches (many
    more image tiles than CTAs), forced on 5,000 images x 2,600 rows of 36,864
    pixels (20 x 11 tiles): sampled images against the FP64 oracle, and the
    same argmins and distances as the contiguous schedule."""
    import torch
    from paper_2109_05339_gb300 import Matcher
    rng = np.random.default_rng(56)
    M, n, P = 2600, 5000, 192
    Y = synth.smooth_rows(rng, M, P)
    pick = rng.integers(0, M, n)
    X = synth.poisson_counts(rng, 0.5 * Y[pick])
    scale = np.float32(2.0)
    Xd, Yd = to_dev(X), to_dev(Y)
    out = {}
    for sched in ("grid", "contiguous"):
        m = Matcher(n, M, P * P, "bf16", 8)
        m.set_schedule(sched)
        m.set_images(Xd, float(scale))
        m.add_slices(Yd)
        out[sched] = {k: v.cpu().numpy() for k, v in m.results().items()}
        m.status()
        m.close()
    del Xd, Yd
    torch.cuda.empty_cache()
    sample = rng.choice(n, 96, replace=False)
    Xs = f32(X[sample]) * np.float64(scale)
    Yf = f32(Y)
    ref = matching.match(Xs, Yf, d=matching.distances_expanded(Xs, Yf))
    ok = ref["margin"] > 1e-4
    assert ok.sum() >= 24
    g = out["grid"]
    np.testing.assert_array_equal(g["best"][sample][ok], ref["best"][ok])
    d_true = np.sum((Xs - Yf[g["best"][sample]]) ** 2, axis=1)
    sc = np.sum(Xs * Xs, 1) + np.sum(Yf[g["best"][sample]] ** 2, 1)
    assert np.all(np.abs(g["d1"][sample] - d_true) <= 1e-5 * sc)
    same = g["best"] == out["contiguous"]["best"]
    assert same.mean() > 0.99
    np.testing.assert_array_equal(g["d1"][same], out["contiguous"]["d1"][same])


@pytest.mark.parametrize("precision,margin", [("bf16", 1e-4), ("fp8", 1e-4)])
def test_c5_matching_rows_of_36864_pixels(precision, margin):
    """1,000 Poisson images against 1,031 model-image-like rows of 192 x 192
    pixels (ragged 256-row tiles, K = 36,864): indices above the margin equal
    the FP64 oracle's, and the returned distance is the exact FP32 distance."""
    import torch
    from paper_2109_05339_gb300 import Matcher
    rng = np.random.default_rng(54)
    M, n, P = 1031, 1000, 192
    Y = synth.smooth_rows(rng, M, P)
    pick = rng.integers(0, M, n)
    X = synth.poisson_counts(rng, 0.5 * Y[pick])
    scale = np.float32(2.0)
    m = Matcher(n, M, P * P, precision, 8)
    m.set_images(to_dev(X), float(scale))
    m.add_slices(to_dev(Y))
    r = {k: v.cpu().numpy() for k, v in m.results().items()}
    m.status()
    m.close()
    torch.cuda.empty_cache()
    Xs = f32(X) * np.float64(scale)
    Yd = f32(Y)
    ref = matching.match(Xs, Yd, d=matching.distances_expanded(Xs, Yd))
    ok = ref["margin"] > margin
    assert ok.sum() >= n // 4
    np.testing.assert_array_equal(r["best"][ok], ref["best"][ok])
    d_true = np.sum((Xs - Yd[r["best"]]) ** 2, axis=1)
    sc = np.sum(Xs * Xs, 1) + np.sum(Yd[r["best"]] ** 2, 1)
    assert np.all(np.abs(r["d1"] - d_true) <= 1e-5 * sc)
