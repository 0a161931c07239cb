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


@pytest.mark.parametrize("cache,chunk", [(True, None), (False, 7)])
def test_iteration_matches_oracle(c1, cache, chunk):
    import torch
    from paper_2109_05339_gb300 import MTIP
    pb, counts, s, ref = c1
    N, P2, M, n = pb.cfg.N, pb.q_lab.shape[0], pb.quats.shape[0], counts.shape[0]
    drv = MTIP(N, 1.0, P2, n, M, orient_chunk=chunk, img_chunk=5 if not cache else None,
               cache_points=cache)
    assert drv.cache_points == cache
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
    if np.all(res["best"].cpu().numpy() == m["best"]):
        assert rel_l2(x.cpu().numpy(), ref["x"]) < 1e-5
    drv.close()
