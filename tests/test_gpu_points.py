"""Point sets (points sorted once for a fixed orientation set): slicing agrees
with spf_slice_model and the oracle; the class-sum merge equals the per-image merge and
the FP64 oracle; orientation chunks accumulate to the whole."""
import numpy as np
import pytest

from oracle import merge, rotation
from tests.gpu_util import f32, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    import torch
    from paper_2109_05339_gb300 import Plan, PointSet
    pb = problem("c1")
    N, P2, M = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0]
    quats = to_dev(pb.quats.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    plan = Plan(N, 1.0, 1e-6, max_points=M * P2)
    ps = PointSet(plan, quats, qlab)
    rng = np.random.default_rng(31)
    images = rng.poisson(8.0, (137, P2)).astype(np.float32)
    images[rng.random(images.shape) < 0.7] = 0.0            # sparse counts, like the c2 images
    best = rng.integers(0, M, 137).astype(np.int32)
    D = (rng.uniform(size=P2) > 0.1).astype(np.float32)
    return dict(pb=pb, plan=plan, ps=ps, quats=quats, qlab=qlab, images=images, best=best, D=D,
                N=N, P2=P2, M=M, torch=torch)


def test_slice_points_matches_slice_model_and_oracle(c1):
    """Point-set slicing (tensor-core interpolation over the sorted bins)
    against the per-call path (CUDA-core gather) and the FP64 oracle."""
    A = to_dev(c1["pb"].A.astype(np.float32))
    a = c1["ps"].slice(A)
    c1["plan"].status()
    b = c1["plan"].slice_model(A, c1["quats"], c1["qlab"])
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 2e-6
    t = rotation.nufft_points(f32(c1["pb"].quats.astype(np.float32)),
                              f32(c1["pb"].q_lab.astype(np.float32)), c1["N"], 1.0).reshape(-1, 3)
    from oracle import nufft
    ref = nufft.type2(f32(c1["pb"].A.astype(np.float32)), t).real.reshape(c1["M"], c1["P2"])
    assert rel_l2(a.cpu().numpy(), ref) < 1e-5


def test_class_sum_merge_equals_per_image_merge_and_oracle(c1):
    torch = c1["torch"]
    plan, ps = c1["plan"], c1["ps"]
    img, best, D = to_dev(c1["images"]), to_dev(c1["best"], torch.int32), to_dev(c1["D"])
    r1, k1 = ps.merge(img, best, D=D, b_scale=0.25)
    r2, k2 = plan.merge_images(img, c1["quats"], c1["qlab"], D=D, b_scale=0.25, orient_idx=best)
    plan.status()
    assert rel_l2(r1.cpu().numpy(), r2.cpu().numpy()) < 1e-6
    assert rel_l2(k1.cpu().numpy(), k2.cpu().numpy()) < 1e-6
    N = c1["N"]
    t = rotation.nufft_points(f32(c1["pb"].quats.astype(np.float32))[c1["best"]],
                              f32(c1["pb"].q_lab.astype(np.float32)), N, 1.0).reshape(-1, 3)
    Dall = np.tile(f32(c1["D"]), len(c1["best"]))
    ref_rhs = merge.rhs(f32(c1["images"]).reshape(-1) * 0.25, t, Dall, N)
    ref_khat = merge.kernel_hat(merge.toeplitz_kernel(t, Dall, N), N)
    assert rel_l2(r1.cpu().numpy(), ref_rhs) < 1e-5
    assert rel_l2(k1.cpu().numpy(), ref_khat) < 1e-5


def test_orientation_chunks_accumulate(c1):
    torch = c1["torch"]
    from paper_2109_05339_gb300 import PointSet
    plan = c1["plan"]
    img, best = to_dev(c1["images"]), to_dev(c1["best"], torch.int32)
    whole_r, whole_k = c1["ps"].merge(img, best, b_scale=0.5)
    rhs = torch.zeros_like(whole_r)
    kh = torch.zeros_like(whole_k)
    for c0, c1_ in [(0, 123), (123, 124), (124, c1["M"])]:
        ps = PointSet(plan, c1["quats"][c0:c1_].contiguous(), c1["qlab"])
        ps.merge(img, best, orient_offset=c0, b_scale=0.5, rhs=rhs, kernel_hat=kh, accumulate=c0 > 0)
        torch.cuda.synchronize()
        ps.close()
    assert rel_l2(rhs.cpu().numpy(), whole_r.cpu().numpy()) < 1e-6
    assert rel_l2(kh.cpu().numpy(), whole_k.cpu().numpy()) < 1e-6
    # images outside every chunk leave the outputs at zero
    empty_r, empty_k = c1["ps"].merge(img, best + c1["M"], b_scale=0.5)
    assert float(empty_r.abs().max()) == 0.0 and float(empty_k.abs().max()) == 0.0


def test_slice_only_set_slices_identically_and_refuses_merge(c1):
    torch = c1["torch"]
    from paper_2109_05339_gb300 import PointSet, SpfError
    A = to_dev(c1["pb"].A.astype(np.float32))
    ps = PointSet(c1["plan"], c1["quats"], c1["qlab"], slice_only=True)
    assert torch.equal(ps.slice(A), c1["ps"].slice(A))
    with pytest.raises(SpfError):
        ps.merge(to_dev(c1["images"]), to_dev(c1["best"], torch.int32))
    ps.close()


def test_dense_point_set_slicing_per_cell_block():
    """A point set dense enough (4,000 orientations of the 16 x 16 detector
    on the 17^3 model: 1.0e6 points, about 700 per 2^3 cell block) that the
    interpolation runs per 2^3 block instead of per 4^3 bin; every output
    against the per-call CUDA-core path, and 4,096 sampled outputs against
    the FP64 direct sum."""
    import torch
    from oracle import nudft
    from paper_2109_05339_gb300 import Plan, PointSet
    pb = problem("c1")
    N = pb.cfg.N
    rng = np.random.default_rng(32)
    q = rng.standard_normal((4000, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = to_dev(q.astype(np.float32))
    qlab = to_dev(pb.q_lab.astype(np.float32))
    P2 = pb.q_lab.shape[0]
    plan = Plan(N, 1.0, 1e-6, max_points=4000 * P2)
    nbins = ((plan.nf + 3) // 4) ** 3
    assert 4000 * P2 >= 256 * 4 * nbins          # the block path's density threshold
    ps = PointSet(plan, quats, qlab)
    A = to_dev(pb.A.astype(np.float32))
    a = ps.slice(A)
    b = plan.slice_model(A, quats, qlab)
    torch.cuda.synchronize()
    plan.status()
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 2e-6
    pick = rng.choice(4000 * P2, 4096, replace=False)
    t = rotation.nufft_points(f32(q.astype(np.float32)), f32(pb.q_lab.astype(np.float32)), N, 1.0).reshape(-1, 3)
    ref = nudft.type2(f32(pb.A.astype(np.float32)), t[pick]).real
    assert rel_l2(a.cpu().numpy().reshape(-1)[pick], ref) < 1e-5
    ps.close()
    plan.close()
