"""Pins of oracle.nufft against the direct sums and independent quadrature."""
import numpy as np
import pytest
from scipy import integrate

from oracle import nudft, nufft


def _points(rng, n, nf):
    t = rng.uniform(-np.pi, np.pi, (n, 3))
    h = 2 * np.pi / nf
    t[0] = [np.pi - 1e-13, -np.pi, 0.0]              # periodic edges
    t[1] = [3 * h, -7 * h, 0.5 * h]                  # exactly on cells / half cells
    t[2] = [np.pi - 0.5 * h, -np.pi + 0.5 * h, 1e-300]
    return t


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N", [5, 9, 13])
def test_type2_type1_match_direct_sums(N):
    rng = np.random.default_rng(N)
    p = nufft.plan(N)
    t = _points(rng, 400, p.nf)
    f = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    v = rng.standard_normal(400) + 1j * rng.standard_normal(400)
    assert _rel(p.type2(f, t), nudft.type2(f, t)) < 1e-9
    assert _rel(p.type1(v, t), nudft.type1(v, t, N)) < 1e-9


def test_exact_transpose():
    rng = np.random.default_rng(21)
    N = 7
    p = nufft.plan(N)
    t = _points(rng, 200, p.nf)
    f = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    v = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    lhs = np.vdot(v, p.type2(f, t))
    rhs = np.vdot(p.type1(v, t), f)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_deconvolution_quadrature_against_adaptive_quadrature():
    w, beta = nufft.es_params(1e-6)
    assert (w, round(beta, 6)) == (7, 16.1)
    nf = nufft.fine_size(17, w)
    assert nf == 36
    p = nufft.deconv_factors(17, nf, w, beta)
    a = w * np.pi / nf
    for k in (0, 3, 8):
        J, _ = integrate.quad(lambda z: float(nufft.phi(z, beta)) * np.cos(k * a * z), -1, 1,
                              epsabs=1e-14, epsrel=1e-13, limit=200)
        assert abs(p[k + 8] - 2.0 / (w * J)) < 1e-11 * abs(p[k + 8])


def test_fine_grid_sizes():
    assert [nufft.fine_size(n, 7) for n in (17, 81, 101, 151, 33, 161, 201, 301)] == \
        [36, 162, 216, 320, 72, 324, 432, 640]


def test_gpu_tolerance_parameters_reach_1e_5():
    """The eps = 1e-6 parameter rule (w = 7) is accurate well inside 1e-5 in FP64."""
    rng = np.random.default_rng(9)
    N = 11
    p = nufft.Plan(N, 1e-6)
    t = _points(rng, 300, p.nf)
    f = rng.standard_normal((N, N, N))
    err = _rel(p.type2(f, t), nudft.type2(f, t))
    assert err < 5e-6
