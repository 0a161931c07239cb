"""Pins of oracle/phasing.py (Sec. II-D) against what the mathematics and the
published methods fix."""
import numpy as np
import pytest

from oracle import phasing


def _blobs(N, centres, widths, weights):
    M = (N - 1) // 2
    d = np.arange(-M, M + 1, dtype=np.float64)
    z, y, x = np.meshgrid(d, d, d, indexing="ij")
    rho = np.zeros((N, N, N))
    for (cx, cy, cz), w, a in zip(centres, widths, weights):
        rho += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * w * w))
    return rho


def test_dft_pair_and_delta_transform():
    rng = np.random.default_rng(1)
    N, M = 9, 4
    rho = rng.standard_normal((N, N, N))
    np.testing.assert_allclose(phasing.idft3(phasing.dft3(rho)).real, rho, atol=1e-12)
    # a delta at n0 transforms to exp(-2 pi i m.n0 / N) (the definition)
    n0 = (2, -3, 1)                                  # (x, y, z)
    delta = np.zeros((N, N, N))
    delta[n0[2] + M, n0[1] + M, n0[0] + M] = 1.0
    m = np.arange(-M, M + 1)
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    ref = np.exp(-2j * np.pi * (mx * n0[0] + my * n0[1] + mz * n0[2]) / N)
    np.testing.assert_allclose(phasing.dft3(delta), ref, atol=1e-12)


def test_modulus_projection_is_a_projection_exact_on_the_data():
    rng = np.random.default_rng(2)
    N = 11
    rho = rng.standard_normal((N, N, N))
    amp = np.abs(phasing.dft3(rng.standard_normal((N, N, N))))
    amp[0, :, :] = -1.0                              # a plane of modes without data
    amp[-1, :, :] = -1.0                             # (its Friedel mates too)
    pm, err = phasing.modulus_projection(rho, amp)
    assert err > 0.1
    F = phasing.dft3(pm)
    data = amp >= 0
    np.testing.assert_allclose(np.abs(F)[data], amp[data], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(F[~data], phasing.dft3(rho)[~data], atol=1e-10)
    pm2, err2 = phasing.modulus_projection(pm, amp)
    np.testing.assert_allclose(pm2, pm, atol=1e-10)
    assert err2 < 1e-12


def test_er_fourier_error_never_increases():
    """Fienup: with the object constraints a projection onto a convex set
    (support and positivity), the ER Fourier error is non-increasing."""
    rng = np.random.default_rng(3)
    N = 15
    rho_true = _blobs(N, [(-2, 1, 0), (1, -1, 2)], [1.2, 1.5], [1.0, 0.7])
    amp = np.abs(phasing.dft3(rho_true))
    support = rho_true > 1e-3 * rho_true.max()
    rho0 = rng.uniform(0, 1, (N, N, N)) * support
    _, _, errs = phasing.run(amp, rho0, support, [("er", 60)])
    assert np.all(np.diff(errs) <= 1e-12 * errs[0])
    assert errs[-1] < errs[0]


def test_hio_er_recover_a_known_object_from_its_magnitudes():
    """A positive object is recovered from its Fourier magnitudes and its own
    support (where it exceeds 1% of its maximum): the support is not
    centrosymmetric, so neither the twin nor a shifted copy fits it."""
    rng = np.random.default_rng(4)
    N = 25
    rho_true = _blobs(N, [(-3, 1, 0), (1, -2, 1), (2, 2, -1)], [1.0, 1.3, 0.9], [1.0, 0.6, 0.8])
    support = rho_true > 1e-2 * rho_true.max()
    assert not np.array_equal(support, support[::-1, ::-1, ::-1])
    rho_true *= support
    amp = np.abs(phasing.dft3(rho_true))
    rho0 = rng.uniform(0, 1, (N, N, N)) * support
    rho, _, errs = phasing.run(amp, rho0, support, [("hio", 1000, 0.9), ("er", 200)])
    assert errs[-1] < 5e-4, errs[-1]
    rel = np.linalg.norm(rho - rho_true) / np.linalg.norm(rho_true)
    assert rel < 1e-2, rel


def test_shrinkwrap_blur_is_a_wrapped_gaussian_filter():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    N, sigma = 13, 1.7
    M = (N - 1) // 2
    rho = rng.standard_normal((N, N, N))
    ref = ndimage.gaussian_filter(np.abs(rho), sigma, mode="wrap", truncate=M / sigma)
    np.testing.assert_allclose(phasing.blur(rho, sigma), ref, atol=1e-12)
    s = phasing.shrinkwrap(rho, sigma, 0.3)
    np.testing.assert_array_equal(s, ref > 0.3 * ref.max())


def test_amplitudes_of_a_circular_autocorrelation():
    """x_n = sum_r rho_r rho_(r+n) (circular, brute force) has DFT |rho^|^2, so
    the amplitudes from the merged model are |rho^|."""
    rng = np.random.default_rng(6)
    N = 7
    rho = rng.uniform(0, 1, (N, N, N))
    x = np.zeros((N, N, N))
    for a in range(N):
        for b in range(N):
            for c in range(N):
                x[a, b, c] = np.sum(rho * np.roll(rho, shift=(-a, -b, -c), axis=(0, 1, 2)))
    # x above is indexed by wrapped offsets; store it centred
    x = np.fft.fftshift(x)
    np.testing.assert_allclose(phasing.amplitudes_from_model(x), np.abs(phasing.dft3(rho)), rtol=1e-10,
                               atol=1e-10)
