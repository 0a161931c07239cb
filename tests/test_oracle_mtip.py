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


def test_model_is_a_fixed_point_of_its_own_noise_free_slices():
    """If the images are the model's own slices at reference orientations
    (here by the direct NUDFT sum, not the oracle's NUFFT), matching recovers
    those orientations exactly, and x = x0 solves the merge's normal equations
    A*DA x + lambda (x - x0) = A*D b (Eq. 2 with b = A x0), so the iteration
    returns the model to the NUFFT's accuracy. A wrong orientation index, image
    scale, weight layout or a right-hand side inconsistent with the Toeplitz
    kernel moves x away from the model."""
    pb = synth.make_problem("c1", n_orient=60, n_img=12)
    rng = np.random.default_rng(7)
    pick = rng.choice(60, 12, replace=False)
    clean = slicing.slice_model(pb.A, pb.quats[pick], pb.q_lab, 1.0, method="direct")
    scale = 0.25
    out = mtip.iteration(pb.A, pb.quats, pb.q_lab, clean / scale, scale, 1.0, cg_iters=6)
    np.testing.assert_array_equal(out["match"]["best"], pick)
    assert np.max(out["match"]["d1"]) < 1e-16 * np.max(out["match"]["d2"])
    x = out["x"]
    assert np.linalg.norm(x - pb.A) < 1e-8 * np.linalg.norm(pb.A)
    assert out["res_hist"][0] < 1e-8 * np.linalg.norm(out["rhs"])
