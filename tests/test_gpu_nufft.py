"""GPU type-2 / type-1 NUFFT (Sec. II-A slicing, Sec. II-C adjoint) against the
FP64 oracle: relative L2 <= 1e-5 at NUFFT tolerance 1e-6, at the same FP32
point coordinates, on sizes spanning several bins and ragged tails."""
import numpy as np
import pytest

from oracle import nudft, nufft, rotation, slicing
from tests.gpu_util import edge_points, f32, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    return T


@pytest.mark.parametrize("N,npts", [(17, 3001), (33, 1999), (5, 77)])
def test_explicit_points_type2_and_type1(torch, N, npts):
    from paper_2109_05339_gb300 import Plan
    rng = np.random.default_rng(N)
    plan = Plan(N, 1.0, 1e-6, max_points=npts)
    t = edge_points(rng, npts, plan.nf)
    A = rng.standard_normal((N, N, N)).astype(np.float32)
    v = rng.standard_normal(npts).astype(np.float32)
    c = plan.nufft_type2(to_dev(A), to_dev(t)).cpu().numpy()
    ref = nudft.type2(f32(A), f32(t)).real
    assert rel_l2(c, ref) < TOL
    f = plan.nufft_type1(to_dev(v), to_dev(t)).cpu().numpy()
    ref1 = nudft.type1(f32(v), f32(t), N).real
    assert rel_l2(f, ref1) < TOL
    # accumulate adds
    f2 = plan.nufft_type1(to_dev(v), to_dev(t), out=to_dev(f), accumulate=True).cpu().numpy()
    assert rel_l2(f2, 2 * ref1) < TOL
    plan.status()


def test_slice_model_c1_matches_oracle(torch):
    from paper_2109_05339_gb300 import Plan
    pb = problem("c1")
    N = pb.cfg.N
    quats = pb.quats.astype(np.float32)
    qlab = pb.q_lab.astype(np.float32)
    A = pb.A.astype(np.float32)
    plan = Plan(N, 1.0, 1e-6, max_points=quats.shape[0] * qlab.shape[0])
    s = plan.slice_model(to_dev(A), to_dev(quats), to_dev(qlab)).cpu().numpy()
    ref = slicing.slice_model(f32(A), f32(quats), f32(qlab), 1.0)
    assert s.shape == ref.shape
    assert rel_l2(s, ref) < TOL
    # the adjoint of the same call
    rng = np.random.default_rng(3)
    g = rng.standard_normal(s.shape).astype(np.float32)
    gA = plan.slice_adjoint(to_dev(g), to_dev(quats), to_dev(qlab)).cpu().numpy()
    refA = slicing.slice_adjoint(f32(g), f32(quats), f32(qlab), N, 1.0)
    assert rel_l2(gA, refA) < TOL
    plan.status()


def test_slice_ragged_and_empty(torch):
    from paper_2109_05339_gb300 import Plan
    pb = problem("c1")
    N = pb.cfg.N
    plan = Plan(N, 1.0, 1e-6, max_points=7 * 37)
    rng = np.random.default_rng(9)
    qlab = (pb.q_lab[rng.choice(256, 37, replace=False)]).astype(np.float32)   # ragged P2
    quats = pb.quats[:7].astype(np.float32)
    A = pb.A.astype(np.float32)
    s = plan.slice_model(to_dev(A), to_dev(quats), to_dev(qlab)).cpu().numpy()
    ref = slicing.slice_model(f32(A), f32(quats), f32(qlab), 1.0, method="direct")
    assert rel_l2(s, ref) < TOL
    empty = plan.slice_model(to_dev(A), to_dev(quats[:0]), to_dev(qlab))
    assert empty.shape == (0, 37)
    z = plan.slice_adjoint(to_dev(np.zeros((0, 37), np.float32)), to_dev(quats[:0]), to_dev(qlab))
    assert float(z.abs().max()) == 0.0
    plan.status()


def test_adjoint_identity_on_device_outputs(torch):
    """<type2 A, v> = <A, type1 v> from GPU outputs, at a larger N."""
    from paper_2109_05339_gb300 import Plan
    N, npts = 41, 50_000
    rng = np.random.default_rng(4)
    plan = Plan(N, 1.0, 1e-6, max_points=npts)
    t = rng.uniform(-np.pi, np.pi, (npts, 3)).astype(np.float32)
    A = rng.standard_normal((N, N, N)).astype(np.float32)
    A = 0.5 * (A + A[::-1, ::-1, ::-1])          # even: type 2 is real
    v = rng.standard_normal(npts).astype(np.float32)
    c = plan.nufft_type2(to_dev(A), to_dev(t)).cpu().numpy().astype(np.float64)
    f = plan.nufft_type1(to_dev(v), to_dev(t)).cpu().numpy().astype(np.float64)
    lhs = float(np.dot(c, v))
    rhs = float(np.sum(A.astype(np.float64) * f))
    assert abs(lhs - rhs) < 1e-5 * np.linalg.norm(c) * np.linalg.norm(v)


def test_plain_nufft_oracle_agrees_at_c1_scale(torch):
    """Sanity link between the two oracle forms used by the larger tests."""
    pb = problem("c1")
    t = rotation.nufft_points(pb.quats[:3], pb.q_lab, pb.cfg.N, 1.0).reshape(-1, 3)
    assert rel_l2(nufft.type2(pb.A, t).real, nudft.type2(pb.A, t).real) < 1e-9


def test_dense_cluster_many_subproblems(torch):
    """Points piled into a few fine cells (like q = 0, where every slice
    passes): one bin holds several subproblems and many points share each tap
    window. Both directions must still match the direct sums."""
    from paper_2109_05339_gb300 import Plan
    N, npts = 17, 20000
    rng = np.random.default_rng(12)
    plan = Plan(N, 1.0, 1e-6, max_points=npts)
    h = 2 * np.pi / plan.nf
    t = np.concatenate([rng.normal(0.0, 0.7 * h, (npts - 2000, 3)),
                        rng.uniform(-np.pi, np.pi, (2000, 3))]).astype(np.float32)
    v = rng.standard_normal(npts).astype(np.float32)
    A = rng.standard_normal((N, N, N)).astype(np.float32)
    f = plan.nufft_type1(to_dev(v), to_dev(t)).cpu().numpy()
    assert rel_l2(f, nudft.type1(f32(v), f32(t), N).real) < TOL
    c = plan.nufft_type2(to_dev(A), to_dev(t)).cpu().numpy()
    assert rel_l2(c, nudft.type2(f32(A), f32(t)).real) < TOL
    plan.status()


def test_slice_chunks_when_sort_buffer_is_small(torch):
    """max_points below M * P2: slicing runs in sorted chunks of whole
    orientations; max_points below P2: unsorted. Same results either way."""
    from paper_2109_05339_gb300 import Plan
    pb = problem("c1")
    N = pb.cfg.N
    quats = pb.quats[:40].astype(np.float32)
    qlab = pb.q_lab.astype(np.float32)
    A = to_dev(pb.A.astype(np.float32))
    ref = slicing.slice_model(f32(pb.A.astype(np.float32)), f32(quats), f32(qlab), 1.0)
    for mp in (40 * 256, 7 * 256 + 3, 100):
        plan = Plan(N, 1.0, 1e-6, max_points=mp)
        s = plan.slice_model(A, to_dev(quats), to_dev(qlab)).cpu().numpy()
        assert rel_l2(s, ref) < TOL, mp
