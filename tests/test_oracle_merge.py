"""Pins of oracle.merge: Toeplitz = direct operator, kernel, CG = dense solve."""
import numpy as np
import pytest

import synth
from oracle import merge, nudft, rotation


def _pts(N, n_img, P, seed):
    rng = np.random.default_rng(seed)
    q = synth.random_quaternions(rng, n_img)
    return rotation.nufft_points(q, synth.detector_qlab(P, 1.0), N, 1.0).reshape(-1, 3), rng


@pytest.mark.parametrize("N", [5, 7])
def test_toeplitz_equals_direct_operator(N):
    t, rng = _pts(N, 6, 8, N)
    D = (rng.uniform(size=t.shape[0]) > 0.1).astype(float)
    x = rng.standard_normal((N, N, N))
    K = merge.toeplitz_kernel(t, D, N)
    Kd = merge.toeplitz_kernel(t, D, N, method="direct")
    assert np.max(np.abs(K - Kd)) < 1e-9 * np.max(np.abs(Kd))
    # K(0) is the diagonal sum of the weights; K is even
    assert abs(Kd[N - 1, N - 1, N - 1] - D.sum()) < 1e-9 * D.sum()
    np.testing.assert_allclose(Kd, Kd[::-1, ::-1, ::-1], atol=1e-9 * D.sum())
    Kh = merge.kernel_hat(K, N)
    assert Kh.shape[0] == merge.embed_size(N)
    y_t = merge.apply_toeplitz(x, Kh, N, lam=0.3)
    y_d = merge.apply_direct(x, t, D, lam=0.3, method="direct")
    assert np.linalg.norm(y_t - y_d) < 1e-9 * np.linalg.norm(y_d)


def test_embed_sizes():
    assert [merge.embed_size(n) for n in (17, 81, 101, 151)] == [36, 162, 216, 320]


def test_rhs_is_linear_over_image_chunks():
    N = 5
    t, rng = _pts(N, 6, 8, 3)
    b = rng.poisson(2.0, t.shape[0]).astype(float)
    D = np.ones(t.shape[0])
    whole = merge.rhs(b, t, D, N)
    half = t.shape[0] // 2
    parts = merge.rhs(b[:half], t[:half], D[:half], N) + merge.rhs(b[half:], t[half:], D[half:], N)
    np.testing.assert_allclose(parts, whole, rtol=1e-12, atol=1e-12 * np.max(np.abs(whole)))
    # and equals Re of the direct adjoint sum
    np.testing.assert_allclose(whole, nudft.type1(b, t, N).real, rtol=1e-8,
                               atol=1e-9 * np.max(np.abs(whole)))


def test_cg_matches_dense_solve():
    N = 5
    t, rng = _pts(N, 4, 6, 4)
    D = np.ones(t.shape[0])
    lam = merge.lambda_from_weights(D, 1e-2)
    n = N ** 3
    H = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        H[:, i] = merge.apply_direct(e.reshape(N, N, N), t, D, lam, method="direct").ravel()
    assert np.allclose(H, H.T, atol=1e-9 * np.max(np.abs(H)))
    assert np.min(np.linalg.eigvalsh(0.5 * (H + H.T))) >= lam * (1 - 1e-9)
    b = rng.poisson(3.0, t.shape[0]).astype(float)
    x0 = rng.standard_normal((N, N, N))
    bt = merge.rhs(b, t, D, N, lam, x0, method="direct")
    x_ref = np.linalg.solve(H, bt.ravel()).reshape(N, N, N)
    Kh = merge.kernel_hat(merge.toeplitz_kernel(t, D, N, method="direct"), N)
    x, hist = merge.cg(lambda v: merge.apply_toeplitz(v, Kh, N, lam), bt, x0, 3 * n)
    assert np.linalg.norm(x - x_ref) < 1e-9 * np.linalg.norm(x_ref)
    # error in the H-norm decreases monotonically
    xs = [x0]
    for k in range(1, 12):
        xs.append(merge.cg(lambda v: merge.apply_toeplitz(v, Kh, N, lam), bt, x0, k)[0])
    en = [float((xk - x_ref).ravel() @ H @ (xk - x_ref).ravel()) for xk in xs]
    assert all(en[i + 1] <= en[i] * (1 + 1e-9) for i in range(len(en) - 1))
