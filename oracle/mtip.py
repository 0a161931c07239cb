"""One slice -> match -> merge -> CG iteration (Fig. 3 without phasing), in FP64.

Used by the tests on small problems and by the CPU baseline on a bounded
sample. Steps, in the paper's order:

1. Slicing (Sec. II-A): model images Re type-2 of A at every orientation.
2. Orientation matching (Sec. II-B): per image the nearest model image.
3. Merging (Sec. II-C, Eq. 2): type-1 of the weighted data (right-hand side)
   and of the weights (Toeplitz kernel), then ``cg_iters`` conjugate-gradient
   steps from x0 = A with lambda = lam_rel * sum(D).

Every part is pinned in its own module; the composition is pinned by the
fixed point that Eq. 2 fixes: images equal to the model's own slices at
reference orientations (direct NUDFT sums) are matched to those orientations
exactly and x = x0 solves the normal equations, so the iteration returns the
model (tests/test_oracle_mtip.py).
"""
import numpy as np

from . import matching, merge, slicing
from .rotation import nufft_points


def iteration(A, quats, q_lab, images, img_scale, qmax, cg_iters, lam_rel=1e-3,
              D=None, k=8, eps=1e-10):
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    P2 = q_lab.shape[0]
    slices = slicing.slice_model(A, quats, q_lab, qmax, eps=eps)
    X = np.asarray(images, dtype=np.float64) * img_scale
    m = matching.match(X, slices, k=k)
    t = nufft_points(np.asarray(quats)[m["best"]], q_lab, N, qmax).reshape(-1, 3)
    Dp = np.ones(P2) if D is None else np.asarray(D, dtype=np.float64)
    Dall = np.tile(Dp, X.shape[0])
    lam = merge.lambda_from_weights(Dall, lam_rel)
    K = merge.toeplitz_kernel(t, Dall, N, eps=eps)
    Kh = merge.kernel_hat(K, N)
    bt = merge.rhs(X.reshape(-1), t, Dall, N, lam, x0=A, eps=eps)
    x, hist = merge.cg(lambda v: merge.apply_toeplitz(v, Kh, N, lam), bt, A, cg_iters)
    return {"slices": slices, "match": m, "K": K, "Khat": Kh, "rhs": bt, "lam": lam,
            "x": x, "res_hist": hist}
