"""Pins of oracle.rotation: known rotations, orthonormality, uniformity, grid mapping."""
import os

import numpy as np

import synth
from oracle import rotation

GOLD = os.path.join(os.path.dirname(__file__), "golden", "rotations_90deg.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        parts = [np.array(p.split(), dtype=float) for p in line.split("|")]
        rows.append(parts)
    return rows


def test_known_rotations():
    for q, ex, ey, ez in _golden():
        R = rotation.quat_to_matrix(q)
        np.testing.assert_allclose(R @ [1, 0, 0], ex, atol=1e-15)
        np.testing.assert_allclose(R @ [0, 1, 0], ey, atol=1e-15)
        np.testing.assert_allclose(R @ [0, 0, 1], ez, atol=1e-15)


def test_orthonormal_det_and_composition():
    rng = np.random.default_rng(5)
    q = synth.random_quaternions(rng, 200)
    R = rotation.quat_to_matrix(q)
    eye = np.einsum("nij,nkj->nik", R, R)
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)
    # Hamilton product q1*q2 corresponds to R1 @ R2.
    a, b = q[0], q[1]
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    prod = np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    np.testing.assert_allclose(rotation.quat_to_matrix(prod), R[0] @ R[1], atol=1e-14)


def test_uniform_mean_rotation_vanishes():
    rng = np.random.default_rng(11)
    R = rotation.quat_to_matrix(synth.random_quaternions(rng, 100_000))
    assert np.max(np.abs(R.mean(axis=0))) < 0.01


def test_grid_points_map_to_dft_frequencies():
    N, qmax = 17, 1.0
    Mh = (N - 1) // 2
    m = np.array([[1, 0, 0], [0, -3, 2], [Mh, Mh, -Mh]], dtype=float)
    ident = np.array([[1.0, 0, 0, 0]])
    t = rotation.nufft_points(ident, m * (qmax / Mh), N, qmax)[0]
    np.testing.assert_allclose(t, 2 * np.pi * m / N, atol=1e-14)
    # every detector point stays inside the periodic band |t| < pi
    qlab = synth.detector_qlab(16, qmax)
    rng = np.random.default_rng(2)
    t = rotation.nufft_points(synth.random_quaternions(rng, 50), qlab, N, qmax)
    assert np.max(np.abs(t)) < np.pi * (N - 1) / N
