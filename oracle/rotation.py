"""Orientations and nonuniform points (Sec. II-A, Table I: q_k).

* ``quat_to_matrix``: active rotation matrix of a unit quaternion (w, x, y, z).
  Pinned by 90-degree rotations about each axis, orthonormality and det = +1.
* ``nufft_points``: t = 2 pi dr R q, the NUFFT coordinates of the rotated
  detector q-points, with dr = 1 / (N dq), dq = qmax / M_h. Grid points
  q = m dq map to t = 2 pi m / N (pinned by the DFT-at-grid-points test).
"""
import numpy as np


def quat_to_matrix(q):
    """Rotation matrices (..., 3, 3) from unit quaternions (..., 4) = (w, x, y, z)."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def radians_per_q(N, qmax):
    """Factor 2 pi dr mapping a physical q to the NUFFT coordinate t."""
    Mh = (N - 1) // 2
    dq = qmax / Mh
    dr = 1.0 / (N * dq)
    return 2.0 * np.pi * dr


def nufft_points(quats, q_lab, N, qmax):
    """t[j, p, :] = 2 pi dr R(quats[j]) q_lab[p], shape (M, P2, 3), float64."""
    R = quat_to_matrix(quats)
    q = np.asarray(q_lab, dtype=np.float64)
    return radians_per_q(N, qmax) * np.einsum("jab,pb->jpa", R, q)
