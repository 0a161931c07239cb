"""Seeded synthetic inputs for the M-TIP slice / match / merge path.

This module is shared by the CPU oracle (through the tests) and by the GPU
product path (through the bench and the tests). It holds no arithmetic of
the method itself: no rotation of points, no NUFFT, no distance and no
solve. It only draws and lays out the inputs:

* a synthetic electron density made of isotropic 3D Gaussians and its
  closed-form diffraction intensity I(q) = |F(q)|^2 (the ground truth the
  model is sampled from; it stands in for the paper's skopi simulation of
  PDB 3IYF, Sec. IV-A, which is not reproduced here);
* the model on the N^3 Cartesian grid (Table I "r" and "q" grids): the
  intensity samples I_m and the autocorrelation coefficients A_n obtained by
  the inverse DFT of those samples;
* reference orientations as unit quaternions, uniform on SO(3);
* the Ewald-sphere q-points of a flat P x P detector;
* Poisson photon counts for given expected-count arrays.

Grid layout: index m in {-M_h..M_h}^3 (M_h = (N-1)/2), stored [z][y][x]
with offset M_h, q_m = m * qmax / M_h. Detector: pitch 1, distance P, the
largest |q| over pixels is 0.9 qmax.

Random draws come from ``numpy.random.Generator(PCG64(seed))`` in a fixed
order: Gaussians (centres, sigmas, weights) -> reference quaternions ->
image orientation picks or off-grid quaternions -> Poisson draws.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Config", "CONFIGS", "Problem", "make_problem", "gaussian_density",
    "intensity_closed_form", "model_grid", "random_quaternions",
    "detector_qlab", "poisson_counts", "smooth_rows", "beamstop_mask",
]


@dataclass(frozen=True)
class Config:
    """One workload shape. Sizes follow the paper's workloads scaled to one GPU."""

    name: str
    seed: int
    n_gauss: int          # Gaussians in the synthetic density
    N: int                # model grid is N^3 (odd)
    P: int                # detector is P x P pixels
    n_orient: int         # reference orientations (model images)
    n_img: int            # experimental images
    photons: float        # c1: per-pixel multiplier; others: mean photons per image
    per_pixel_scale: bool  # True: lambda = photons * slice; False: global fluence s
    images_on_grid: bool  # True: images at reference orientations; False: off-grid
    cg_iters: int
    qmax: float = 1.0
    eps: float = 1e-6     # NUFFT tolerance of the GPU path


CONFIGS = {
    # 12 Gaussians, 17^3, 16x16, 500 orientations, 100 images at reference
    # orientations, x1e3 per pixel then Poisson, one CG step.
    "c1": Config("c1", 1, 12, 17, 16, 500, 100, 1e3, True, True, 1),
    # 200 Gaussians, 81^3, 128x128, 1e4 x 1e4, mean 1e3 photons/image, 10 CG.
    "c2": Config("c2", 2, 200, 81, 128, 10_000, 10_000, 1e3, False, False, 10),
    # precision study on c1 shapes
    "c3": Config("c3", 3, 12, 17, 16, 500, 100, 1e3, True, True, 1),
    # differentiation: 101^3, 128x128, 5e4 images at known quaternions
    "c4": Config("c4", 4, 200, 101, 128, 0, 50_000, 1e3, False, False, 20),
    # full iteration at the largest one-GPU size
    "c5": Config("c5", 5, 200, 151, 192, 100_000, 100_000, 5e2, False, False, 10),
}


def gaussian_density(rng: np.random.Generator, n: int):
    """Centres uniform in the radius-0.3 ball, sigma ~ U[0.03, 0.08], weights ~ U[0.5, 1]."""
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 0.3 * rng.random(n) ** (1.0 / 3.0)
    centres = d * r[:, None]
    sigmas = rng.uniform(0.03, 0.08, n)
    weights = rng.uniform(0.5, 1.0, n)
    return centres, sigmas, weights


def intensity_closed_form(q, centres, sigmas, weights, chunk: int = 4096):
    """Ground-truth intensity |F(q)|^2 of the Gaussian density at q (..., 3).

    rho(r) = sum_j w_j (2 pi s_j^2)^(-3/2) exp(-|r - c_j|^2 / (2 s_j^2)) has
    F(q) = sum_j w_j exp(-2 pi^2 s_j^2 |q|^2) exp(-2 pi i q.c_j).
    """
    q = np.asarray(q, dtype=np.float64)
    shp = q.shape[:-1]
    qf = q.reshape(-1, 3)
    out = np.empty(qf.shape[0])
    for s in range(0, qf.shape[0], chunk):
        qq = qf[s:s + chunk]
        q2 = np.sum(qq * qq, axis=1)
        env = np.exp(-2.0 * np.pi ** 2 * np.outer(q2, sigmas ** 2)) * weights
        ph = -2.0 * np.pi * (qq @ centres.T)
        F = np.sum(env * np.exp(1j * ph), axis=1)
        out[s:s + chunk] = F.real ** 2 + F.imag ** 2
    return out.reshape(shp)


def model_grid(N: int, qmax: float, centres, sigmas, weights):
    """Intensity samples I_m and autocorrelation coefficients A_n on the N^3 grid.

    Grid index m = (m_x, m_y, m_z) in {-M_h..M_h}^3, M_h = (N-1)/2, stored as
    [m_z + M_h][m_y + M_h][m_x + M_h]; q_m = m * qmax / M_h. A_n is the inverse
    DFT  A_n = N^-3 sum_m I_m exp(+2 pi i m.n / N), real and even because I is
    real and Friedel-even; it is returned as float64 with the same layout.
    """
    assert N % 2 == 1
    Mh = (N - 1) // 2
    ax = np.arange(-Mh, Mh + 1) * (qmax / Mh)
    qz, qy, qx = np.meshgrid(ax, ax, ax, indexing="ij")
    q = np.stack([qx, qy, qz], axis=-1)
    I = intensity_closed_form(q, centres, sigmas, weights)
    # numpy's ifftn uses exp(+2 pi i k n / N) / N^3; shift centred <-> wrapped.
    A = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(I))).real
    return I, np.ascontiguousarray(A)


def random_quaternions(rng: np.random.Generator, n: int):
    """Unit quaternions (w, x, y, z), uniform on SO(3), sign fixed so w >= 0."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def detector_qlab(P: int, qmax: float, edge_frac: float = 0.9):
    """Ewald-sphere q-points of a flat P x P detector, shape (P*P, 3), float64.

    Pixel pitch 1, sample-detector distance P, pixel (a, b) centred at
    (a - (P-1)/2, b - (P-1)/2, P); flattened index b*P + a. q = (s_hat - z_hat)
    / wavelength, with the wavelength chosen so that the largest |q| over all
    pixels (a corner pixel) is edge_frac * qmax.
    """
    c = np.arange(P) - (P - 1) / 2.0
    b, a = np.meshgrid(c, c, indexing="ij")
    pix = np.stack([a.ravel(), b.ravel(), np.full(P * P, float(P))], axis=1)
    s = pix / np.linalg.norm(pix, axis=1, keepdims=True)
    d = s - np.array([0.0, 0.0, 1.0])
    wavelength = np.max(np.linalg.norm(d, axis=1)) / (edge_frac * qmax)
    return d / wavelength


def beamstop_mask(P: int, radius: float):
    """Pixel weights of a P x P detector with a beam stop: 0 for pixels whose
    centre lies within `radius` pixels of the detector centre, 1 elsewhere
    (float32, flattened b*P + a like detector_qlab)."""
    c = np.arange(P) - (P - 1) / 2.0
    b, a = np.meshgrid(c, c, indexing="ij")
    return (np.hypot(a, b).ravel() > radius).astype(np.float32)


def poisson_counts(rng: np.random.Generator, lam):
    """Poisson photon counts with the given expectations (float32 output)."""
    return rng.poisson(np.maximum(np.asarray(lam, dtype=np.float64), 0.0)).astype(np.float32)


def smooth_rows(rng: np.random.Generator, n: int, P: int, n_blobs: int = 24, width=(4.0, 20.0)):
    """n smooth non-negative P x P images (rows of length P*P, float32): each a
    random positive combination of isotropic 2D Gaussian blobs on the pixel
    grid. Used as model-image-like rows where a test needs many of them
    without computing slices."""
    yy, xx = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    cx = rng.uniform(0, P, n_blobs)
    cy = rng.uniform(0, P, n_blobs)
    sw = rng.uniform(width[0], width[1], n_blobs)
    basis = np.exp(-((xx[None] - cx[:, None, None]) ** 2 + (yy[None] - cy[:, None, None]) ** 2)
                   / (2 * sw[:, None, None] ** 2)).reshape(n_blobs, P * P)
    coef = rng.gamma(1.0, 1.0, (n, n_blobs))
    return (coef @ basis).astype(np.float32)


@dataclass
class Problem:
    """All seeded inputs of one configuration except the photon counts."""

    cfg: Config
    centres: np.ndarray
    sigmas: np.ndarray
    weights: np.ndarray
    I_grid: np.ndarray        # (N,N,N) float64 intensity samples
    A: np.ndarray             # (N,N,N) float64 autocorrelation coefficients
    quats: np.ndarray         # (n_orient, 4) float64 reference orientations
    q_lab: np.ndarray         # (P*P, 3) float64
    img_pick: np.ndarray | None   # (n_img,) int indices into quats (on-grid images)
    img_quats: np.ndarray     # (n_img, 4) float64 orientation of each image
    rng: np.random.Generator = field(repr=False)

    def image_counts(self, noise_free_slices):
        """Poisson photon counts for the images, from their noise-free slices.

        ``noise_free_slices`` (n_img, P*P) are the model slices at the image
        orientations, computed by whichever side builds the test. Returns
        (counts float32, scale s) where the expected counts are s * slice.
        For per-pixel-scale configs s = photons; otherwise s makes the mean
        photons per image equal to cfg.photons.
        """
        sl = np.asarray(noise_free_slices, dtype=np.float64)
        s = self.fluence(sl)
        return poisson_counts(self.rng, s * sl), s

    def fluence(self, noise_free_slices) -> float:
        if self.cfg.per_pixel_scale:
            return float(self.cfg.photons)
        tot = np.mean(np.sum(np.asarray(noise_free_slices, dtype=np.float64), axis=1))
        return float(self.cfg.photons / tot)


def make_problem(cfg: Config | str, n_orient: int | None = None, n_img: int | None = None) -> Problem:
    """Draw every seeded input of ``cfg`` (optionally with fewer orientations/images).

    Overriding n_orient / n_img keeps the draw order, so a smaller problem is
    a prefix-consistent variant only for the Gaussians; the quaternion draws
    change with the counts.
    """
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    M = cfg.n_orient if n_orient is None else n_orient
    Ni = cfg.n_img if n_img is None else n_img
    rng = np.random.Generator(np.random.PCG64(cfg.seed))
    centres, sigmas, weights = gaussian_density(rng, cfg.n_gauss)
    I_grid, A = model_grid(cfg.N, cfg.qmax, centres, sigmas, weights)
    quats = random_quaternions(rng, M) if M > 0 else np.zeros((0, 4))
    if cfg.images_on_grid and M > 0:
        pick = rng.integers(0, M, Ni)
        img_quats = quats[pick]
    else:
        pick = None
        img_quats = random_quaternions(rng, Ni)
    q_lab = detector_qlab(cfg.P, cfg.qmax)
    return Problem(cfg, centres, sigmas, weights, I_grid, A, quats, q_lab, pick, img_quats, rng)
