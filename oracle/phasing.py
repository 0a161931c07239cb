"""Phasing (Sec. II-D): from the merged diffraction volume to a density.

TEST INFRASTRUCTURE ONLY (see the package header).

Starting from a seed state, real-space constraints on rho and reciprocal-space
constraints on its transform are applied in turn: error reduction (ER,
Gerchberg-Saxton as analysed by Fienup), hybrid input-output (HIO, Fienup) and
shrinkwrap support updates (Marchesini), the published methods the paper
cites. This module writes them out on the model's own N^3 grid (N odd,
index n in {-M..M}^3 stored [n_z+M][n_y+M][n_x+M]):

  transform      rho^_m = sum_n rho_n exp(-2 pi i m.n / N)        (dft3)
                 rho_n  = N^-3 sum_m rho^_m exp(+2 pi i m.n / N)  (idft3)
  data           amp_m = sqrt(max(I_m, 0)) with I_m = Re dft3(x)_m the
                 intensity of the merged autocorrelation x (x_n =
                 N^-3 sum_m I_m exp(+2 pi i m.n / N) is the circular
                 autocorrelation of rho when I = |rho^|^2); amp_m < 0 marks
                 a mode without data (left free)
  P_M (modulus)  rho^ -> amp rho^ / |rho^| on modes with data (amp when
                 rho^ = 0), unchanged elsewhere; back to real space, real part
  ER             rho' = P_M rho where (support and, with positivity,
                 P_M rho > 0), else 0
  HIO            rho' = P_M rho where (support and, with positivity,
                 P_M rho > 0), else rho - beta P_M rho
  Fourier error  E_F(rho) = sqrt(sum_data (|rho^| - amp)^2 / sum_data amp^2)
  shrinkwrap     blur = |rho| circularly convolved with the normalised
                 Gaussian g(d) ~ exp(-|d|^2 / (2 sigma^2)), d over the
                 minimal periodic images {-M..M}^3; support = blur >
                 threshold * max(blur)

Pins (tests): the DFT pair and a delta's transform; P_M idempotent and
exact on the data; the ER Fourier error non-increasing (Fienup's result);
recovery of a known non-centrosymmetric object from its magnitudes with its
support; the shrinkwrap blur against scipy's wrapped Gaussian filter; the
amplitudes of a brute-force circular autocorrelation.
"""
import numpy as np


def dft3(rho):
    """rho^_m = sum_n rho_n exp(-2 pi i m.n / N), centred storage in and out."""
    return np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(np.asarray(rho))))


def idft3(F):
    """rho_n = N^-3 sum_m F_m exp(+2 pi i m.n / N), centred storage in and out."""
    return np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(np.asarray(F))))


def amplitudes_from_model(x):
    """Measured Fourier magnitudes from the merged autocorrelation x."""
    I = dft3(np.asarray(x, dtype=np.float64)).real
    return np.sqrt(np.maximum(I, 0.0))


def modulus_projection(rho, amp):
    """P_M rho (real part) and the Fourier error of rho."""
    F = dft3(np.asarray(rho, dtype=np.float64))
    mag = np.abs(F)
    data = amp >= 0
    unit = np.where(mag > 0, F / np.where(mag > 0, mag, 1.0), 1.0)
    Fp = np.where(data, amp * unit, F)
    num = float(np.sum((mag[data] - amp[data]) ** 2))
    den = float(np.sum(amp[data] ** 2))
    return idft3(Fp).real, np.sqrt(num / den) if den > 0 else 0.0


def _keep(pm, support, positivity):
    return support & (pm > 0) if positivity else support.copy()


def er_step(rho, amp, support, positivity=True):
    pm, err = modulus_projection(rho, amp)
    return np.where(_keep(pm, support, positivity), pm, 0.0), err


def hio_step(rho, amp, support, beta=0.9, positivity=True):
    pm, err = modulus_projection(rho, amp)
    return np.where(_keep(pm, support, positivity), pm, rho - beta * pm), err


def gaussian_kernel(N, sigma):
    """Normalised Gaussian on the minimal periodic offsets {-M..M}^3 (centred)."""
    M = (N - 1) // 2
    d = np.arange(-M, M + 1, dtype=np.float64)
    g1 = np.exp(-d * d / (2.0 * sigma * sigma))
    g = g1[:, None, None] * g1[None, :, None] * g1[None, None, :]
    return g / g.sum()


def blur(rho, sigma):
    """|rho| circularly convolved with the normalised Gaussian kernel."""
    N = np.asarray(rho).shape[0]
    G = dft3(gaussian_kernel(N, sigma))
    return idft3(dft3(np.abs(rho)) * G).real


def shrinkwrap(rho, sigma, threshold):
    b = blur(rho, sigma)
    return b > threshold * b.max()


def run(amp, rho0, support0, schedule, positivity=True):
    """Apply a schedule of steps: ("er", n), ("hio", n, beta), ("shrinkwrap",
    sigma, threshold). Returns (rho, support, Fourier errors of every ER/HIO
    iterate before its step)."""
    rho = np.array(rho0, dtype=np.float64, copy=True)
    support = np.array(support0, dtype=bool, copy=True)
    errs = []
    for step in schedule:
        kind = step[0]
        if kind == "er":
            for _ in range(step[1]):
                rho, e = er_step(rho, amp, support, positivity)
                errs.append(e)
        elif kind == "hio":
            for _ in range(step[1]):
                rho, e = hio_step(rho, amp, support, step[2], positivity)
                errs.append(e)
        elif kind == "shrinkwrap":
            support = shrinkwrap(rho, step[1], step[2])
        else:
            raise ValueError(kind)
    return rho, support, np.array(errs)
