"""Pins of oracle.lcurve: residual via normal-equation quantities equals the
direct type-2 residual; exact Tikhonov solutions trace a monotone L-curve;
the curvature formula finds the known corner of an analytic curve."""
import numpy as np

import synth
from oracle import lcurve, merge, nudft, rotation


def _problem(seed=3, N=5):
    rng = np.random.default_rng(seed)
    q = synth.random_quaternions(rng, 4)
    t = rotation.nufft_points(q, synth.detector_qlab(6, 1.0), N, 1.0).reshape(-1, 3)
    D = (rng.uniform(size=t.shape[0]) > 0.2).astype(float)
    b = rng.poisson(3.0, t.shape[0]).astype(float)
    return rng, t, D, b, N


def test_toeplitz_residual_equals_direct():
    rng, t, D, b, N = _problem()
    x = rng.standard_normal((N, N, N))
    K = merge.toeplitz_kernel(t, D, N, method="direct")
    Kh = merge.kernel_hat(K, N)
    rhs = merge.rhs(b, t, D, N, method="direct")
    direct = lcurve.residual_norm2(x, t, D, b, method="direct")
    via = lcurve.residual_norm2_toeplitz(x, Kh, rhs, float(np.sum(D * b * b)))
    assert abs(via - direct) < 1e-9 * direct


def test_exact_solutions_trace_monotone_curve():
    rng, t, D, b, N = _problem(4)
    n = N ** 3
    lams = np.logspace(-3, 2, 9) * D.sum() * 1e-2
    K = merge.toeplitz_kernel(t, D, N, method="direct")
    Kh = merge.kernel_hat(K, N)
    rhs = merge.rhs(b, t, D, N, method="direct")
    x0 = np.zeros((N, N, N))
    res, reg = [], []
    for lam in lams:
        H = np.empty((n, n))
        for i in range(n):
            e = np.zeros(n)
            e[i] = 1.0
            H[:, i] = merge.apply_toeplitz(e.reshape(N, N, N), Kh, N, lam).ravel()
        x = np.linalg.solve(H, rhs.ravel()).reshape(N, N, N)
        res.append(lcurve.residual_norm2(x, t, D, b, method="direct"))
        reg.append(float(np.sum(x * x)))
    assert all(np.diff(res) >= -1e-9 * np.max(res))      # residual grows with lambda
    assert all(np.diff(reg) <= 1e-9 * np.max(reg))       # penalty shrinks with lambda


def test_curvature_finds_the_corner_of_an_analytic_l():
    # (rho, eta) along a smoothed L: a hyperbola-like curve with its corner at s = 0
    s = np.linspace(-4, 4, 33)
    rho = np.log1p(np.exp(2 * s))       # flat for s < 0, rising for s > 0
    eta = np.log1p(np.exp(-2 * s))      # falling for s < 0, flat for s > 0
    lams = np.exp(s)
    idx = lcurve.corner(lams, np.exp(2 * rho), np.exp(2 * eta))
    assert abs(s[idx]) < 0.3
    # hand check of the three-point derivative on an uneven grid: exact for quadratics
    ss = np.array([0.0, 0.3, 1.0, 1.2, 2.0])
    y = 3 * ss ** 2 - ss + 1
    np.testing.assert_allclose(lcurve._d1(y, ss), 6 * ss[1:-1] - 1, rtol=1e-12)
    np.testing.assert_allclose(lcurve._d2(y, ss), np.full(3, 6.0), rtol=1e-12)
