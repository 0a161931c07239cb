"""Merging (Sec. II-C): Tikhonov normal equations (Eq. 2) solved by CG.

Eq. 2 is  A* D A x + lambda (x - x0) = A* D b. With real model coefficients x
and real intensities b, the real normal equations are

    H x = b~,   H = Re(A^H D A) + lambda I,   b~ = Re(A^H D b) + lambda x0,

where (A x)_j = sum_n x_n exp(-i n.t_j) (type 2) and A^H is type 1.

* ``toeplitz_kernel``: (Re A^H D A x)_n = sum_n' K(n - n') x_n' with
  K(d) = Re sum_j D_j exp(+i d.t_j) on d in {-(N-1)..N-1}^3: a type-1 NUFFT with
  the data replaced by the weights ("type-1 with ones" when D = 1).
* ``kernel_hat``: circulant embedding of K in P_T^3 (P_T = smallest even
  2/3/5-smooth >= 2N-1) and its FFT; real because K is real and even.
* ``apply_toeplitz``: zero-pad x to P_T^3, FFT, multiply by K^, inverse FFT,
  crop: the Toeplitz product (Fessler), then + lambda x.
* ``apply_direct``: Re(type1(D * type2(x))) + lambda x, one forward and one
  adjoint NUFFT (Sec. III-A); pinned equal to the Toeplitz form.
* ``rhs``: b~ = Re(type1(D b)) + lambda x0.
* ``cg``: textbook conjugate gradient from x0 for a fixed number of steps,
  pinned against numpy.linalg.solve on a dense H.
* ``lambda_from_weights``: lambda = lam_rel * sum_j D_j (sum_j D_j is the
  diagonal of Re A^H D A).
"""
import numpy as np

from . import nudft, nufft


def embed_size(N):
    """Smallest even 2/3/5-smooth integer >= 2N - 1."""
    n = 2 * N - 1
    n += n % 2
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 2


def _type1(v, t, n_modes, method, eps):
    if method == "direct":
        return nudft.type1(v, t, n_modes)
    return nufft.type1(v, t, n_modes, eps)


def _type2(x, t, method, eps):
    if method == "direct":
        return nudft.type2(x, t)
    return nufft.type2(x, t, eps)


def toeplitz_kernel(t, D, N, method="nufft", eps=1e-10):
    """K(d) = Re sum_j D_j exp(+i d.t_j), shape (2N-1,)*3 stored [d_z][d_y][d_x]."""
    return _type1(np.asarray(D, dtype=np.float64), t, 2 * N - 1, method, eps).real


def _wrap(N, PT):
    Mh = (N - 1) // 2
    return np.arange(-Mh, Mh + 1) % PT


def kernel_hat(K, N, PT=None):
    """FFT of the circulant embedding of K (2N-1)^3 in PT^3; real array."""
    PT = embed_size(N) if PT is None else PT
    Kc = np.zeros((PT, PT, PT))
    ix = np.arange(-(N - 1), N) % PT
    Kc[np.ix_(ix, ix, ix)] = K
    return np.fft.fftn(Kc).real


def apply_toeplitz(x, Khat, N, lam=0.0):
    PT = Khat.shape[0]
    xp = np.zeros((PT, PT, PT))
    ix = _wrap(N, PT)
    xp[np.ix_(ix, ix, ix)] = x
    y = np.fft.ifftn(np.fft.fftn(xp) * Khat).real
    return y[np.ix_(ix, ix, ix)] + lam * x


def apply_direct(x, t, D, lam=0.0, method="nufft", eps=1e-10):
    N = x.shape[0]
    Ax = _type2(x, t, method, eps)
    return _type1(np.asarray(D) * Ax, t, N, method, eps).real + lam * x


def rhs(b, t, D, N, lam=0.0, x0=None, method="nufft", eps=1e-10):
    v = np.asarray(D, dtype=np.float64) * np.asarray(b, dtype=np.float64).reshape(-1)
    out = _type1(v, t, N, method, eps).real
    if x0 is not None:
        out = out + lam * x0
    return out


def lambda_from_weights(D, lam_rel=1e-3):
    return float(lam_rel * np.sum(np.asarray(D, dtype=np.float64)))


def cg(apply_H, btilde, x0, iters):
    """Conjugate gradient on H x = btilde from x0; returns x and |r_k| history."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = btilde - apply_H(x)
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    hist = [np.sqrt(rr)]
    for _ in range(iters):
        Ap = apply_H(p)
        alpha = rr / float(np.vdot(p, Ap).real)
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.vdot(r, r).real)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        hist.append(np.sqrt(rr))
    return x, np.array(hist)
