"""Plain exponential-of-semicircle (ES) NUFFT, step by step (FP64).

The paper computes slicing with a type-2 NUFFT and merging with type-1 NUFFTs
(Sec. II-A, II-C, III-A), using the FINUFFT/cuFINUFFT libraries it cites. This
module restates that published method in plain NumPy:

  kernel        phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, else 0,
                width w = ceil(log10(1/eps)) + 1 fine-grid cells, beta = 2.30 w,
                upsampling sigma = 2, fine grid n_f = smallest even 2/3/5-smooth
                integer >= max(2 N_modes, 2 w), spacing h = 2 pi / n_f.
  correction    psi(x) = phi(x / a), a = w h / 2, has Fourier transform
                psi^(k) = a int_{-1}^{1} phi(z) cos(k a z) dz (Gauss-Legendre).
                Per axis the deconvolution factor is p_k = h / psi^(k)
                            = 2 / (w int_{-1}^{1} phi(z) cos(k a z) dz).
  type 2        1. g[k mod n_f] = f_k p_kx p_ky p_kz (zero elsewhere)
                2. G_l = sum_k g_k exp(-2 pi i k.l / n_f)        (numpy fftn)
                3. c_j = sum over the w^3 cells l nearest to u_j = t_j / h of
                         G_l phi((l_x-u_x) 2/w) phi((l_y-u_y) 2/w) phi((l_z-u_z) 2/w),
                   cell indices taken mod n_f.
  type 1        the exact transpose: spread v_j with the same weights onto the
                fine grid b, F_k = sum_l b_l exp(+2 pi i k.l / n_f), f_k = F_k p_k...

Default tolerance here is eps = 1e-10 (w = 11), far below the GPU path's 1e-6,
so that the oracle's own error does not blur parity. Pinned against the
direct sums in ``nudft`` (relative L2 error and adjoint identity) and the
quadrature against scipy's adaptive quadrature.
"""
import math

import numpy as np


def es_params(eps):
    """Kernel width w (cells) and shape beta for tolerance eps, upsampling 2."""
    w = int(math.ceil(math.log10(1.0 / eps))) + 1
    return w, 2.30 * w


def phi(z, beta):
    """ES kernel on z in [-1, 1] (zero outside)."""
    z = np.asarray(z, dtype=np.float64)
    inside = np.abs(z) <= 1.0
    s = np.sqrt(np.where(inside, 1.0 - z * z, 0.0))
    return np.where(inside, np.exp(beta * (s - 1.0)), 0.0)


def fine_size(n_modes, w):
    """Smallest even 2/3/5-smooth integer >= max(2 n_modes, 2 w)."""
    n = max(2 * n_modes, 2 * w)
    n += n % 2
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 2


def deconv_factors(n_modes, nf, w, beta, n_quad=256):
    """p_k = 2 / (w int_{-1}^{1} phi(z) cos(k a z) dz) for k = -M..M, a = w pi / nf."""
    Mh = (n_modes - 1) // 2
    k = np.arange(-Mh, Mh + 1, dtype=np.float64)
    z, wq = np.polynomial.legendre.leggauss(n_quad)
    a = w * np.pi / nf
    J = (wq * phi(z, beta)) @ np.cos(np.outer(z, k) * a)
    return 2.0 / (w * J)


class Plan:
    """Plain NUFFT set-up for an N_modes^3 mode cube."""

    def __init__(self, n_modes, eps=1e-10):
        assert n_modes % 2 == 1
        self.n_modes = n_modes
        self.w, self.beta = es_params(eps)
        self.nf = fine_size(n_modes, self.w)
        self.p = deconv_factors(n_modes, self.nf, self.w, self.beta)

    # -- shared pieces -------------------------------------------------------
    def _mode_index(self):
        Mh = (self.n_modes - 1) // 2
        return np.arange(-Mh, Mh + 1) % self.nf

    def _taps(self, t):
        """Flat fine-grid indices (n, w, w, w) and weights (n, w, w, w) of points t."""
        w, nf = self.w, self.nf
        u = np.asarray(t, dtype=np.float64) * (nf / (2.0 * np.pi))
        l0 = np.ceil(u - w / 2.0)
        cells = l0[:, :, None] + np.arange(w)[None, None, :]          # (n, 3, w)
        wts = phi((cells - u[:, :, None]) * (2.0 / w), self.beta)
        idx = np.mod(cells, nf).astype(np.int64)
        flat = (idx[:, 2, :, None, None] * nf * nf + idx[:, 1, None, :, None] * nf
                + idx[:, 0, None, None, :])
        wprod = wts[:, 2, :, None, None] * wts[:, 1, None, :, None] * wts[:, 0, None, None, :]
        return flat, wprod

    def _chunk(self):
        return max(1, (1 << 22) // self.w ** 3)

    # -- type 2 ----------------------------------------------------------------
    def fine_grid(self, f):
        """Steps 1-2 of type 2: the deconvolved, zero-padded modes and their
        FFT, G_l = sum_k g_k exp(-2 pi i k.l / n_f), flattened (n_f^3,)."""
        nf = self.nf
        f = np.asarray(f)
        assert f.shape == (self.n_modes,) * 3
        g = np.zeros((nf, nf, nf), dtype=np.complex128)
        ix = self._mode_index()
        pz, py, px = np.meshgrid(self.p, self.p, self.p, indexing="ij")
        g[np.ix_(ix, ix, ix)] = f * (pz * py * px)
        return np.fft.fftn(g).ravel()

    def interp(self, G, t):
        """Step 3 of type 2: c_j = sum over the w^3 nearest cells of G_l times
        the three kernel weights, for points t (npts, 3)."""
        t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
        out = np.empty(t.shape[0], dtype=np.complex128)
        cs = self._chunk()
        for s in range(0, t.shape[0], cs):
            flat, wprod = self._taps(t[s:s + cs])
            out[s:s + cs] = np.sum(G[flat] * wprod, axis=(1, 2, 3))
        return out

    def type2(self, f, t):
        """c_j = sum_n f_n exp(-i n.t_j) (approximately); f (M,M,M), t (npts, 3)."""
        return self.interp(self.fine_grid(f), t)

    # -- type 1 ----------------------------------------------------------------
    def spread(self, v, t):
        """Fine-grid b_l = sum_j v_j psi(x_l - t_j) (complex, (nf, nf, nf))."""
        nf = self.nf
        v = np.asarray(v).reshape(-1).astype(np.complex128)
        t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
        bre = np.zeros(nf ** 3)
        bim = np.zeros(nf ** 3)
        cs = self._chunk()
        for s in range(0, t.shape[0], cs):
            flat, wprod = self._taps(t[s:s + cs])
            vv = v[s:s + cs][:, None, None, None]
            bre += np.bincount(flat.ravel(), weights=(vv.real * wprod).ravel(), minlength=nf ** 3)
            bim += np.bincount(flat.ravel(), weights=(vv.imag * wprod).ravel(), minlength=nf ** 3)
        return (bre + 1j * bim).reshape(nf, nf, nf)

    def modes_of(self, b):
        """Last steps of type 1: F_k = sum_l b_l exp(+2 pi i k.l / n_f) of the
        spread grid b, kept for the n_modes^3 modes and deconvolved."""
        nf = self.nf
        F = np.fft.ifftn(b) * float(nf) ** 3          # sum_l b_l exp(+2 pi i k.l / nf)
        ix = self._mode_index()
        pz, py, px = np.meshgrid(self.p, self.p, self.p, indexing="ij")
        return F[np.ix_(ix, ix, ix)] * (pz * py * px)

    def type1(self, v, t):
        """f_n = sum_j v_j exp(+i n.t_j) (approximately) for the n_modes^3 modes."""
        return self.modes_of(self.spread(v, t))


_PLANS = {}


def plan(n_modes, eps=1e-10):
    key = (n_modes, eps)
    if key not in _PLANS:
        _PLANS[key] = Plan(n_modes, eps)
    return _PLANS[key]


def type2(f, t, eps=1e-10):
    return plan(np.asarray(f).shape[0], eps).type2(f, t)


def type1(v, t, n_modes, eps=1e-10):
    return plan(n_modes, eps).type1(v, t)
