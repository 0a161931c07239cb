"""L-curve choice of the Tikhonov parameter (Sec. II-C: each rank solves with a
different regularisation parameter and the L-curve selects the solution).

For each lambda in a sweep the merge solve gives x_lambda; the curve is
(rho, eta) = (log |A x - b|_D, log |x - x0|) and the chosen lambda is where
its curvature, as a function of log lambda, is largest:

  kappa = (rho' eta'' - rho'' eta') / (rho'^2 + eta'^2)^(3/2),

derivatives by finite differences on the (possibly uneven) log lambda grid,
interior points only.

* ``residual_norm2``: |A x - b|_D^2 = sum_j D_j |(A x)_j - b_j|^2 with the
  complex type-2 transform, written out.
* ``residual_norm2_toeplitz``: the same from the normal-equation quantities,
  x.T x - 2 x.rhs + b.D b with T = Re(A^H D A) and rhs = Re(A^H D b);
  pinned equal to the direct form.
* ``corner``: the maximum-curvature index.
"""
import numpy as np

from . import merge, nudft, nufft


def residual_norm2(x, t, D, b, method="nufft", eps=1e-10):
    Ax = nudft.type2(x, t) if method == "direct" else nufft.type2(x, t, eps)
    r = Ax - np.asarray(b, dtype=np.float64)
    return float(np.sum(np.asarray(D, dtype=np.float64) * (r.real ** 2 + r.imag ** 2)))


def residual_norm2_toeplitz(x, Khat, rhs_data, b_norm2):
    N = x.shape[0]
    Tx = merge.apply_toeplitz(x, Khat, N, 0.0)
    return float(np.sum(x * Tx) - 2.0 * np.sum(x * rhs_data) + b_norm2)


def _d1(y, s):
    """First derivative at interior points on an uneven grid (three-point)."""
    h0 = s[1:-1] - s[:-2]
    h1 = s[2:] - s[1:-1]
    return (-(h1 / (h0 * (h0 + h1))) * y[:-2] + ((h1 - h0) / (h0 * h1)) * y[1:-1]
            + (h0 / (h1 * (h0 + h1))) * y[2:])


def _d2(y, s):
    h0 = s[1:-1] - s[:-2]
    h1 = s[2:] - s[1:-1]
    return 2.0 * (y[:-2] / (h0 * (h0 + h1)) - y[1:-1] / (h0 * h1) + y[2:] / (h1 * (h0 + h1)))


def curvature(lams, res2, reg2):
    """kappa at the interior points of the curve (log residual, log penalty)."""
    s = np.log(np.asarray(lams, dtype=np.float64))
    rho = 0.5 * np.log(np.asarray(res2, dtype=np.float64))
    eta = 0.5 * np.log(np.asarray(reg2, dtype=np.float64))
    r1, r2 = _d1(rho, s), _d2(rho, s)
    e1, e2 = _d1(eta, s), _d2(eta, s)
    return (r1 * e2 - r2 * e1) / (r1 * r1 + e1 * e1) ** 1.5


def corner(lams, res2, reg2):
    """Index (into lams) of the maximum-curvature point."""
    return int(np.argmax(curvature(lams, res2, reg2))) + 1


def sweep(t, D, b, N, x0, lams, iters, eps=1e-10):
    """CG solve per lambda; returns (x list, res2, reg2, corner index)."""
    K = merge.toeplitz_kernel(t, D, N, eps=eps)
    Kh = merge.kernel_hat(K, N)
    rhs_data = merge.rhs(b, t, D, N, eps=eps)
    b_norm2 = float(np.sum(np.asarray(D) * np.asarray(b, dtype=np.float64) ** 2))
    xs, res2, reg2 = [], [], []
    for lam in lams:
        x, _ = merge.cg(lambda v: merge.apply_toeplitz(v, Kh, N, lam), rhs_data + lam * x0, x0, iters)
        xs.append(x)
        res2.append(residual_norm2_toeplitz(x, Kh, rhs_data, b_norm2))
        reg2.append(float(np.sum((x - x0) ** 2)))
    return xs, np.array(res2), np.array(reg2), corner(lams, res2, reg2)
