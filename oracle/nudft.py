"""Direct non-uniform DFT sums -- the definitions of Sec. II-A and II-C.

Modes n = (n_x, n_y, n_z) in {-M_h..M_h}^3 for a (N, N, N) array stored
[n_z][n_y][n_x] with offset M_h; points t_j = (t_x, t_y, t_z) in radians.

* type 2 (slicing, "uniform to nonuniform"):  c_j = sum_n f_n exp(-i n.t_j)
* type 1 (the adjoint, merging):               f_n = sum_j v_j exp(+i n.t_j)

Each sum is evaluated literally, one exponential per (point, mode) pair, in
FP64. Pins (tests): at grid points t = 2 pi m / N type 2 equals numpy's DFT;
<type2 f, v> = <f, type1 v>; brute-force triple loops on N = 3; the Gaussian
closed form.
"""
import numpy as np


def mode_vectors(N):
    """All modes n as an (N^3, 3) array (x, y, z) in storage order."""
    Mh = (N - 1) // 2
    k = np.arange(-Mh, Mh + 1)
    nz, ny, nx = np.meshgrid(k, k, k, indexing="ij")
    return np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=1).astype(np.float64)


def _chunk(N, budget=2 ** 22):
    return max(1, budget // (N ** 3))


def type2(f, t):
    """c_j = sum_n f_n exp(-i n.t_j); f (N,N,N) real or complex, t (npts, 3)."""
    f = np.asarray(f)
    N = f.shape[0]
    n = mode_vectors(N)
    fv = f.reshape(-1).astype(np.complex128)
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.complex128)
    cs = _chunk(N)
    for s in range(0, t.shape[0], cs):
        ph = t[s:s + cs] @ n.T
        out[s:s + cs] = np.exp(-1j * ph) @ fv
    return out


def type1(v, t, N):
    """f_n = sum_j v_j exp(+i n.t_j) for the N^3 modes; returns complex (N,N,N)."""
    n = mode_vectors(N)
    v = np.asarray(v).reshape(-1).astype(np.complex128)
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(n.shape[0], dtype=np.complex128)
    cs = _chunk(N)
    for s in range(0, t.shape[0], cs):
        ph = t[s:s + cs] @ n.T
        out += v[s:s + cs] @ np.exp(1j * ph)
    return out.reshape(N, N, N)


def type1_modes(v, t, modes):
    """f_n for a given list of modes (K, 3) only: the definition at sampled outputs."""
    modes = np.asarray(modes, dtype=np.float64).reshape(-1, 3)
    v = np.asarray(v).reshape(-1).astype(np.complex128)
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(modes.shape[0], dtype=np.complex128)
    cs = 1 << 20
    for s in range(0, t.shape[0], cs):
        ph = t[s:s + cs] @ modes.T
        out += v[s:s + cs] @ np.exp(1j * ph)
    return out
