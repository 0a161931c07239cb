"""Slicing (Sec. II-A), its adjoint, and the gradient of the slice loss.

* ``slice_model``: model image j, pixel p = Re c(t_jp), c the type-2 sum of the
  real autocorrelation coefficients A at t_jp = 2 pi dr R_j q_p. For real, even
  A the imaginary part vanishes (Friedel symmetry, pinned by a test).
* ``slice_adjoint``: gradA_n = Re sum_{j,p} g_jp exp(+i n.t_jp) (type 1), the
  transpose of ``slice_model`` (pinned by the inner-product identity).
* ``loss`` / ``loss_grad``: L(A) = 1/2 sum (slice_model(A) - b)^2 and its
  gradient Re(type1(slice_model(A) - b)). L is quadratic in A, so central
  finite differences are exact up to rounding (pinned by a test).
"""
import numpy as np

from . import nudft, nufft
from .rotation import nufft_points


def _type2(A, t, method, eps):
    if method == "direct":
        return nudft.type2(A, t)
    return nufft.type2(A, t, eps)


def _type1(v, t, N, method, eps):
    if method == "direct":
        return nudft.type1(v, t, N)
    return nufft.type1(v, t, N, eps)


def slice_model(A, quats, q_lab, qmax, method="nufft", eps=1e-10):
    """Model images (M, P2) float64 of the (N,N,N) model A at quaternions (M, 4)."""
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    t = nufft_points(quats, q_lab, N, qmax)
    M, P2 = t.shape[:2]
    return _type2(A, t.reshape(-1, 3), method, eps).real.reshape(M, P2)


def slice_adjoint(g, quats, q_lab, N, qmax, method="nufft", eps=1e-10):
    """gradA (N,N,N) = Re type-1 of g (M, P2) at the same points."""
    t = nufft_points(quats, q_lab, N, qmax).reshape(-1, 3)
    return _type1(np.asarray(g, dtype=np.float64).reshape(-1), t, N, method, eps).real


def loss(A, quats, q_lab, b, qmax, method="nufft", eps=1e-10):
    r = slice_model(A, quats, q_lab, qmax, method, eps) - np.asarray(b, dtype=np.float64)
    return 0.5 * float(np.sum(r * r))


def loss_grad(A, quats, q_lab, b, qmax, method="nufft", eps=1e-10):
    N = np.asarray(A).shape[0]
    r = slice_model(A, quats, q_lab, qmax, method, eps) - np.asarray(b, dtype=np.float64)
    return slice_adjoint(r, quats, q_lab, N, qmax, method, eps)
