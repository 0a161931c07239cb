"""16-bit photon-count images: the device conversion is exact (aligned
vector path, unaligned scalar path, ragged tails, counts above 32767 carried
in int16), and an M-TIP iteration fed counts equals the one fed the same
images as FP32 (the same argmins; the merged model up to the order of
floating-point atomic sums)."""
import numpy as np
import pytest

import synth
from tests.gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,offset", [(0, 0), (7, 0), (8, 0), (1003, 0), (1 << 20, 0), (1003, 1), (4096, 3)])
def test_counts_to_f32_exact(n, offset):
    import torch
    from paper_2109_05339_gb300 import counts_to_f32
    rng = np.random.default_rng(n + offset)
    vals = rng.integers(0, 65536, n + offset, dtype=np.int64)
    vals[: min(3, n + offset)] = [0, 65535, 32768][: min(3, n + offset)]
    buf = torch.from_numpy(vals.astype(np.uint16).view(np.int16)).cuda()
    src = buf[offset:]                       # offset > 0: not 16-byte aligned
    out = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    counts_to_f32(src, out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), vals[offset:].astype(np.float32))


def test_iteration_from_counts_equals_fp32():
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb = synth.make_problem("c1", n_orient=60, n_img=12)
    from oracle import slicing
    clean = slicing.slice_model(pb.A, pb.img_quats, pb.q_lab, 1.0, method="direct")
    # Poisson frames at a mean of 50 photons per pixel: counts fit 16 bits
    s = 50.0 / float(np.mean(clean))
    counts = np.random.default_rng(5).poisson(np.maximum(clean, 0.0) * s).astype(np.float32)
    assert counts.max() <= 65535
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    A = to_dev(pb.A.astype(np.float32))
    q = to_dev(pb.quats.astype(np.float32))
    lab = to_dev(pb.q_lab.astype(np.float32))
    out = []
    for as_counts in (False, True):
        drv = MTIP(N, 1.0, P2, n, M, cache_points=True)
        imgs = to_dev(counts.astype(np.float32))
        if as_counts:
            imgs = torch.from_numpy(counts.astype(np.uint16).view(np.int16)).cuda()
        res, x, lam = drv.iteration(A, q, lab, imgs, 1.0 / s, cg_iters=3)
        torch.cuda.synchronize()
        out.append((res["best"].cpu().numpy(), x.cpu().numpy().copy(), lam))
        drv.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    # the merge sums with floating-point atomics: equal up to summation order
    assert rel_l2(out[1][1], out[0][1]) < 1e-6
    assert out[0][2] == out[1][2]
