"""Pins of oracle.nudft: brute force, DFT at grid points, adjoint, Gaussian closed forms."""
import itertools

import numpy as np

import synth
from oracle import nudft, rotation


def test_bruteforce_loops_N3():
    rng = np.random.default_rng(1)
    N = 3
    f = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    t = rng.uniform(-np.pi, np.pi, (7, 3))
    v = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    c_ref = np.zeros(7, dtype=complex)
    g_ref = np.zeros((N, N, N), dtype=complex)
    for j in range(7):
        for iz, iy, ix in itertools.product(range(N), repeat=3):
            nx, ny, nz = ix - 1, iy - 1, iz - 1
            ph = nx * t[j, 0] + ny * t[j, 1] + nz * t[j, 2]
            c_ref[j] += f[iz, iy, ix] * complex(np.cos(ph), -np.sin(ph))
            g_ref[iz, iy, ix] += v[j] * complex(np.cos(ph), np.sin(ph))
    np.testing.assert_allclose(nudft.type2(f, t), c_ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(nudft.type1(v, t, N), g_ref, rtol=1e-13, atol=1e-13)


def test_grid_points_equal_numpy_dft_and_return_I():
    pb = synth.make_problem("c1", n_orient=1, n_img=1)
    N = pb.cfg.N
    Mh = (N - 1) // 2
    m = nudft.mode_vectors(N)
    t = rotation.nufft_points(np.array([[1.0, 0, 0, 0]]), m * (pb.cfg.qmax / Mh), N, pb.cfg.qmax)[0]
    c = nudft.type2(pb.A, t)
    I = pb.I_grid.ravel()
    assert np.max(np.abs(c - I)) < 1e-13 * np.max(I)
    # and against numpy's forward DFT of a random complex cube
    rng = np.random.default_rng(3)
    f = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    ref = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(f)))
    np.testing.assert_allclose(nudft.type2(f, t), ref.ravel(), rtol=1e-12, atol=1e-11)


def test_adjoint_identity():
    rng = np.random.default_rng(4)
    N = 7
    f = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    t = rng.uniform(-np.pi, np.pi, (300, 3))
    v = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    lhs = np.vdot(v, nudft.type2(f, t))
    rhs = np.vdot(nudft.type1(v, t, N), f)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def _gauss3(r2, s2):
    return (2 * np.pi * s2) ** -1.5 * np.exp(-r2 / (2 * s2))


def test_gaussian_closed_forms_pin_sign_and_scale():
    """type 2 of a finely sampled Gaussian density (and of its autocorrelation)
    equals the continuous Fourier transform F(q) (and |F(q)|^2)."""
    rng = np.random.default_rng(7)
    centres, _, weights = synth.gaussian_density(rng, 3)
    sigmas = np.array([0.05, 0.065, 0.08])
    h = 1.0 / 32
    half = int(np.ceil(1.5 / h))
    N = 2 * half + 1
    ax = np.arange(-half, half + 1) * h
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    rho = np.zeros_like(x)
    acf = np.zeros_like(x)
    for j in range(3):
        rho += weights[j] * _gauss3((x - centres[j, 0]) ** 2 + (y - centres[j, 1]) ** 2
                                    + (z - centres[j, 2]) ** 2, sigmas[j] ** 2)
        for l in range(3):
            d = centres[l] - centres[j]
            acf += weights[j] * weights[l] * _gauss3(
                (x - d[0]) ** 2 + (y - d[1]) ** 2 + (z - d[2]) ** 2, sigmas[j] ** 2 + sigmas[l] ** 2)
    q = rng.uniform(-1, 1, (20, 3))
    t = 2 * np.pi * h * q
    F_ref = np.sum(weights * np.exp(-2 * np.pi ** 2 * np.outer(np.sum(q * q, 1), sigmas ** 2))
                   * np.exp(-2j * np.pi * q @ centres.T), axis=1)
    F = h ** 3 * nudft.type2(rho, t)
    np.testing.assert_allclose(F, F_ref, rtol=1e-10, atol=1e-12)
    I = h ** 3 * nudft.type2(acf, t)
    np.testing.assert_allclose(I.real, np.abs(F_ref) ** 2, rtol=1e-10)
    assert np.max(np.abs(I.imag)) < 1e-10 * np.max(np.abs(F_ref) ** 2)
    # the generator's closed form agrees with the same ground truth
    np.testing.assert_allclose(synth.intensity_closed_form(q, centres, sigmas, weights),
                               np.abs(F_ref) ** 2, rtol=1e-13)


def test_type1_modes_matches_full():
    rng = np.random.default_rng(8)
    N = 5
    t = rng.uniform(-np.pi, np.pi, (100, 3))
    v = rng.standard_normal(100)
    full = nudft.type1(v, t, N).ravel()
    modes = nudft.mode_vectors(N)
    pick = [0, 17, 62, 124]
    np.testing.assert_allclose(nudft.type1_modes(v, t, modes[pick]), full[pick], rtol=1e-13)
