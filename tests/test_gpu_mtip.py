"""The M-TIP driver's whole iteration (slice -> match -> merge -> CG) against
the oracle's iteration, with point sets kept across iterations, with only
their slicing sort kept (image chunks merged at their matched orientations),
and streamed per orientation chunk (the modes for orientation sets too large
to keep sorted; ragged chunks): same matches above the margin, same merged
model."""
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
                                              (False, 9, True), ("slices", 7, False), ("slices", 9, True)])
def test_iteration_matches_oracle(c1, cache, chunk, keep):
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    drv = MTIP(N, 1.0, P2, n, M, orient_chunk=chunk, img_chunk=5 if cache is not True else None,
               cache_points=cache, keep_slices=keep)
    assert drv.point_mode == {True: "cached", False: "streamed", "slices": "slice sets kept"}[cache]
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


@pytest.mark.parametrize("budget,mode", [(300_000, "cached"), (100_000, "slice sets kept"),
                                         (30_000, "streamed")])
def test_point_mode_follows_the_budget(c1, budget, mode):
    """Left to choose, the driver keeps full point sets (16 B per orientation x
    pixel) when they fit the budget, else slice-only sets (4 B), else streams:
    60 orientations x 256 pixels take 245,760 B full and 61,440 B slice-only."""
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    drv = MTIP(N, 1.0, P2, n, M, point_budget_bytes=budget)
    assert drv.point_mode == mode
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


def test_repeated_iterations_reuse_zeroed_class_sums(c1):
    """Kept point sets: each merge spreads only the nonzero class sums and
    leaves them zeroed, so the next iteration forms its sums without a
    clearing pass. Three iterations on the same inputs give the same matches
    and, up to the order of atomic additions, the same model as the first
    and as the oracle."""
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    drv = MTIP(N, 1.0, P2, n, M, orient_chunk=25, cache_points=True)
    args = (to_dev(pb.A.astype(np.float32)), to_dev(pb.quats.astype(np.float32)),
            to_dev(pb.q_lab.astype(np.float32)), to_dev(counts.astype(np.float32)), 1.0 / s)
    outs = []
    for _ in range(3):
        res, x, lam = drv.iteration(*args, cg_iters=3)
        torch.cuda.synchronize()
        outs.append((res["best"].cpu().numpy(), x.cpu().numpy().copy()))
    drv.plan.status()
    for best, x in outs[1:]:
        np.testing.assert_array_equal(best, outs[0][0])
        assert rel_l2(x, outs[0][1]) < 1e-6
    # a fourth merge (at the oracle's argmins) on the sums left zeroed
    x2, _ = drv.solve(*args, torch.as_tensor(ref["match"]["best"], dtype=torch.int32, device="cuda"), cg_iters=3)
    torch.cuda.synchronize()
    assert rel_l2(x2.cpu().numpy(), ref["x"]) < 1e-5
    drv.close()


@pytest.mark.parametrize("mode,pinned", [("sm", True), ("copy", True), ("sm", False)])
def test_host_buffer_iteration_equals_device_iteration(c1, mode, pinned):
    """The iteration from host buffers (16-bit counts; page-locked images read
    by the SMs or moved by the copy engines, or pageable images, which take
    the copy engines in either mode) gives the matches and the merged model
    of the iteration on device buffers, call after call (the two input slots
    alternate)."""
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    # 16-bit counts (the c1 images hold up to about 9e4 photons a pixel: halved)
    c16 = np.floor(counts / 2).astype(np.uint16)
    assert c16.max() > 32767 and c16.max() == np.floor(counts.max() / 2)   # the top bit is used and kept
    q = to_dev(pb.quats.astype(np.float32))
    ql = to_dev(pb.q_lab.astype(np.float32))
    drv = MTIP(N, 1.0, P2, n, M, cache_points=True, host_images="u16")
    drv.set_orientations(q, ql)
    drv.set_upload(mode)
    A_h = torch.from_numpy(pb.A.astype(np.float32))
    img_h = torch.from_numpy(c16.view(np.int16))
    if pinned:
        A_h, img_h = A_h.pin_memory(), img_h.pin_memory()
    outs = []
    for _ in range(3):
        best, x, lam = drv.iteration_host(A_h, img_h, 2.0 / s, cg_iters=3)
        torch.cuda.synchronize()
        outs.append((best.numpy().copy(), x.numpy().copy(), lam))
    assert drv.last_upload_ms() >= 0.0
    res, xd, lamd = drv.iteration(to_dev(pb.A.astype(np.float32)), q, ql, to_dev(c16.astype(np.float32)),
                                  2.0 / s, cg_iters=3)
    torch.cuda.synchronize()
    drv.status()
    for best, x, lam in outs:
        np.testing.assert_array_equal(best, res["best"].cpu().numpy())
        assert lam == lamd
        assert rel_l2(x, xd.cpu().numpy()) < 1e-6
    drv.close()
