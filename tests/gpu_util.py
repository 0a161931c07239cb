"""Shared helpers of the GPU parity tests (inputs from synth, expectations from oracle)."""
import functools

import numpy as np

import synth


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32(x):
    """The FP32 value both sides receive, as float64 for the oracle."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@functools.lru_cache(maxsize=None)
def problem(name, n_orient=None, n_img=None):
    return synth.make_problem(name, n_orient=n_orient, n_img=n_img)


def to_dev(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x), dtype=dtype or torch.float32)
    return t.cuda()


def edge_points(rng, n, nf):
    """Random points in radians plus periodic edges and cell / half-cell points."""
    t = rng.uniform(-np.pi, np.pi, (n, 3))
    h = 2 * np.pi / nf
    t[0] = [np.pi - 1e-6, -np.pi, 0.0]
    t[1] = [3 * h, -7 * h, 0.5 * h]
    t[2] = [np.pi - 0.5 * h, -np.pi + 0.5 * h, 1e-30]
    t[3] = [7.5, -9.0, 2 * np.pi]            # outside [-pi, pi): taken mod 2 pi
    return t.astype(np.float32)
