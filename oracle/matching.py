"""Orientation matching (Sec. II-B): nearest model image in Euclidean distance.

* ``distances``: d_ij = sum_p (x_ip - y_jp)^2 in FP64, the plain definition,
  image by image.
* ``distances_expanded``: |x_i|^2 + |y_j|^2 - 2 x_i.y_j with an FP64 matmul;
  used only where the plain form is too slow, and pinned against it.
* ``match``: per image the argmin over orientations (ties go to the lowest
  orientation index), the best and second-best distances d1 <= d2, the top-k
  orientation indices in (distance, index) order, and the relative margin
  m_i = (d2 - d1) / (|x_i|^2 + |y_best|^2) together with (d2 - d1) / d2.
* Optional pixel weights D (e.g. 0 behind the beam stop, Sec. II-C):
  d_ij = sum_p D_p (x_ip - y_jp)^2, norms weighted the same way.
"""
import numpy as np


def _weights(D, n):
    return np.ones(n) if D is None else np.asarray(D, dtype=np.float64)


def distances(X, Y, D=None):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    w = _weights(D, X.shape[1])
    d = np.empty((X.shape[0], Y.shape[0]))
    for i in range(X.shape[0]):
        diff = Y - X[i][None, :]
        d[i] = np.sum(w[None, :] * diff * diff, axis=1)
    return d


def distances_expanded(X, Y, D=None):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    w = _weights(D, X.shape[1])
    x2 = np.sum(w * X * X, axis=1)
    y2 = np.sum(w * Y * Y, axis=1)
    return x2[:, None] + y2[None, :] - 2.0 * ((X * w) @ Y.T)


def topk_lowest(d, k):
    """Indices of the k smallest entries per row; ties broken by lower index."""
    order = np.argsort(d, axis=1, kind="stable")
    return order[:, :k]


def match(X, Y, k=8, d=None, D=None):
    """Matching results of images X (Ni, P2) against model images Y (M, P2)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if d is None:
        d = distances(X, Y, D)
    top = topk_lowest(d, max(k, 2))
    rows = np.arange(d.shape[0])
    best = top[:, 0]
    d1 = d[rows, best]
    d2 = d[rows, top[:, 1]] if d.shape[1] > 1 else np.full(d.shape[0], np.inf)
    w = _weights(D, X.shape[1])
    x2 = np.sum(w * X * X, axis=1)
    y2 = np.sum(w * Y * Y, axis=1)
    margin = (d2 - d1) / (x2 + y2[best])
    with np.errstate(divide="ignore", invalid="ignore"):
        margin_alt = np.where(d2 > 0, (d2 - d1) / d2, 0.0)
    return {"best": best, "d1": d1, "d2": d2, "topk": top[:, :k], "margin": margin,
            "margin_alt": margin_alt, "d": d}
