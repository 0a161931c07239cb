"""The oracle's full iteration on c1 recovers the generating orientations and
its CG lowers the residual; the merged model moves towards the truth."""
import numpy as np

import synth
from oracle import mtip, slicing


def test_c1_iteration():
    pb = synth.make_problem("c1", n_orient=60, n_img=12)
    clean = slicing.slice_model(pb.A, pb.img_quats, pb.q_lab, 1.0, method="direct")
    counts, s = pb.image_counts(clean)
    out = mtip.iteration(pb.A, pb.quats, pb.q_lab, counts, 1.0 / s, 1.0, cg_iters=3)
    m = out["match"]
    ok = m["margin"] > 1e-3
    np.testing.assert_array_equal(m["best"][ok], pb.img_pick[ok])
    assert out["res_hist"][-1] < out["res_hist"][0]
