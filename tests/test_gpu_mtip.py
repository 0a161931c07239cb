"""The M-TIP driver's whole iteration (slice -> match -> merge -> CG) against
the oracle's iteration, with point sets kept across iterations and streamed
per orientation chunk (the mode for orientation sets too large to keep
sorted; ragged chunks): same matches above the margin, same merged model."""
import numpy as np
import pytest

import synth
from oracle import mtip, slicing
from tests.gpu_util import f32, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    pb = synth.make_problem("c1", n_orient=60, n_img=12)
    clean = slicing.slice_model(pb.A, pb.img_quats, pb.q_lab, 1.0, method="direct")
    counts, s = pb.image_counts(clean)
    A32 = f32(pb.A.astype(np.float32))
    q32 = f32(pb.quats.astype(np.float32))
    l32 = f32(pb.q_lab.astype(np.float32))
    ref = mtip.iteration(A32, q32, l32, counts, 1.0 / s, 1.0, cg_iters=3)
    return pb, counts, s, ref


@pytest.mark.parametrize("cache,chunk,keep", [(True, None, None), (False, 7, False), (True, 7, True),
                                              (False, 9, True)])
def test_iteration_matches_oracle(c1, cache, chunk, keep):
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    drv = MTIP(N, 1.0, P2, n, M, orient_chunk=chunk, img_chunk=5 if not cache else None,
               cache_points=cache, keep_slices=keep)
    assert drv.cache_points == cache
    if keep is not None:
        assert drv.keep_slices == keep
    res, x, lam = drv.iteration(to_dev(pb.A.astype(np.float32)), to_dev(pb.quats.astype(np.float32)),
                                to_dev(pb.q_lab.astype(np.float32)), to_dev(counts.astype(np.float32)),
                                1.0 / s, cg_iters=3)
    torch.cuda.synchronize()
    drv.plan.status()
    m = ref["match"]
    ok = m["margin"] > 1e-4
    assert ok.sum() >= n // 2
    np.testing.assert_array_equal(res["best"].cpu().numpy()[ok], m["best"][ok])
    assert abs(lam - ref["lam"]) <= 1e-9 * ref["lam"]
    # the merged volume, always compared: merge and solve at the oracle's
    # argmins (images below the margin may legitimately match elsewhere)
    x2, lam2 = drv.solve(to_dev(pb.A.astype(np.float32)), to_dev(pb.quats.astype(np.float32)),
                         to_dev(pb.q_lab.astype(np.float32)), to_dev(counts.astype(np.float32)), 1.0 / s,
                         torch.as_tensor(m["best"], dtype=torch.int32, device="cuda"), cg_iters=3)
    torch.cuda.synchronize()
    drv.plan.status()
    assert lam2 == lam
    assert rel_l2(x2.cpu().numpy(), ref["x"]) < 1e-5
    if np.all(res["best"].cpu().numpy() == m["best"]):
        assert rel_l2(x.cpu().numpy(), ref["x"]) < 1e-5
    drv.close()


def test_orientation_set_rewritten_in_place_is_taken_again(c1):
    """A caller who rewrites the quaternion tensor in place gets slices of the
    new orientations: the driver keys its sorted point sets on the tensor's
    in-place version, not only on its address."""
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    drv = MTIP(N, 1.0, P2, n, M, cache_points=True)
    A = to_dev(pb.A.astype(np.float32))
    q = to_dev(pb.quats.astype(np.float32))
    ql = to_dev(pb.q_lab.astype(np.float32))
    imgs = to_dev(counts.astype(np.float32))
    drv.iteration(A, q, ql, imgs, 1.0 / s, cg_iters=1)
    q.copy_(q.flip(0))                                  # same storage, new contents
    res, _, _ = drv.iteration(A, q, ql, imgs, 1.0 / s, cg_iters=1)
    torch.cuda.synchronize()
    fresh = MTIP(N, 1.0, P2, n, M, cache_points=True)
    res2, _, _ = fresh.iteration(A, q.clone(), ql, imgs, 1.0 / s, cg_iters=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(res["best"].cpu().numpy(), res2["best"].cpu().numpy())
    drv.close()
    fresh.close()


def test_iteration_with_a_process_group_equals_without(c1):
    """The image-sharded driver path on one rank (gloo group of size 1): the
    merge's sums go through the group reduction and lambda through the
    global count; the result equals the driver without a group."""
    import socket
    import torch
    import torch.distributed as dist
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    dist.init_process_group("gloo", rank=0, world_size=1, init_method=f"tcp://127.0.0.1:{port}")
    try:
        out = []
        for group in (None, dist.group.WORLD):
            drv = MTIP(N, 1.0, P2, n, M, cache_points=True, process_group=group)
            res, x, lam = drv.iteration(to_dev(pb.A.astype(np.float32)), to_dev(pb.quats.astype(np.float32)),
                                        to_dev(pb.q_lab.astype(np.float32)), to_dev(counts.astype(np.float32)),
                                        1.0 / s, cg_iters=3)
            torch.cuda.synchronize()
            out.append((res["best"].cpu().numpy(), x.cpu().numpy().copy(), lam))
            drv.close()
    finally:
        dist.destroy_process_group()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][2] == out[1][2]
    assert rel_l2(out[1][1], out[0][1]) < 1e-6
