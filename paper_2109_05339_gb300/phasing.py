"""Phasing (Sec. II-D): ER, HIO and shrinkwrap on the model grid, run by the
library (spf_phaser_* in include/spf.h). This module marshals tensors and
runs a schedule of steps; every transform, projection and error sum is a
library kernel."""
from __future__ import annotations

import ctypes as C

import torch

from ._lib import SPF_PHASE_ER, SPF_PHASE_HIO, check, lib
from .api import _dev_index, _f32, _ptr, _stream


class Phaser:
    """Phasing state on an N^3 grid: iterate, support, magnitudes."""

    def __init__(self, N: int, device=None):
        self.device = _dev_index(device)
        h = C.c_void_p()
        check(lib.spf_phaser_create(C.byref(h), int(N), self.device))
        self._h = h
        self.N = int(N)

    def close(self):
        if getattr(self, "_h", None):
            lib.spf_phaser_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cube(self, t, name):
        return _f32(t, name, self.device, (self.N,) * 3)

    def set_amplitudes(self, amp):
        """Fourier magnitudes (N^3, centred storage; < 0: no data)."""
        check(lib.spf_phaser_set_amplitudes(self._h, _ptr(self._cube(amp, "amp")), _stream(self.device)))

    def amplitudes_from_model(self, x):
        """Magnitudes sqrt(max(I, 0)) of a merged autocorrelation x."""
        check(lib.spf_phaser_amplitudes_from_model(self._h, _ptr(self._cube(x, "x")), _stream(self.device)))

    def set_state(self, rho=None, support=None):
        if rho is not None:
            self._cube(rho, "rho")
        if support is not None:
            if support.dtype not in (torch.uint8, torch.bool) or tuple(support.shape) != (self.N,) * 3 \
                    or not support.is_contiguous() or support.device.index != self.device:
                raise ValueError("support must be a contiguous uint8/bool (N, N, N) tensor on the phaser's device")
        check(lib.spf_phaser_set_state(self._h, _ptr(rho), _ptr(support), _stream(self.device)))

    def iterate(self, method, iters, beta=0.9, positivity=True, errors=None):
        """`iters` ER or HIO steps; errors: float64 device tensor (iters,) or None."""
        m = {"er": SPF_PHASE_ER, "hio": SPF_PHASE_HIO}[method]
        if errors is not None and (errors.dtype != torch.float64 or errors.numel() < iters):
            raise ValueError("errors must be a float64 device tensor of iters values")
        check(lib.spf_phaser_iterate(self._h, m, int(iters), C.c_float(beta), int(bool(positivity)), _ptr(errors),
                                     _stream(self.device)))

    def shrinkwrap(self, sigma, threshold):
        check(lib.spf_phaser_shrinkwrap(self._h, C.c_float(sigma), C.c_float(threshold), _stream(self.device)))

    def get(self):
        """(rho, support as uint8, magnitudes) as new device tensors."""
        d = torch.device("cuda", self.device)
        rho = torch.empty((self.N,) * 3, dtype=torch.float32, device=d)
        sup = torch.empty((self.N,) * 3, dtype=torch.uint8, device=d)
        amp = torch.empty((self.N,) * 3, dtype=torch.float32, device=d)
        check(lib.spf_phaser_get(self._h, _ptr(rho), _ptr(sup), _ptr(amp), _stream(self.device)))
        return rho, sup, amp

    def run(self, schedule, positivity=True):
        """Apply ("er", n), ("hio", n, beta) and ("shrinkwrap", sigma,
        threshold) steps in order; returns the Fourier errors of every ER/HIO
        iterate (float64 device tensor)."""
        n = sum(st[1] for st in schedule if st[0] in ("er", "hio"))
        errs = torch.zeros(max(n, 1), dtype=torch.float64, device=torch.device("cuda", self.device))
        k = 0
        for st in schedule:
            if st[0] == "er":
                self.iterate("er", st[1], positivity=positivity, errors=errs[k:k + st[1]])
                k += st[1]
            elif st[0] == "hio":
                self.iterate("hio", st[1], beta=st[2], positivity=positivity, errors=errs[k:k + st[1]])
                k += st[1]
            elif st[0] == "shrinkwrap":
                self.shrinkwrap(st[1], st[2])
            else:
                raise ValueError(st[0])
        return errs[:n]
