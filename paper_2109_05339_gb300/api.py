"""PyTorch-facing wrappers of the C ABI (include/spf.h).

PyTorch provides device memory and the current CUDA stream; every step of
slicing, matching and merging runs in the library's CUDA kernels. The
wrappers check shapes and dtypes, then pass raw pointers and sizes.
"""
from __future__ import annotations

import ctypes as C

import torch

from ._lib import SPF_BF16, SPF_FP8, SPF_FP32, SpfError, check, lib

__all__ = ["Plan", "PointSet", "Matcher", "SliceModel", "slice_model", "counts_to_f32", "SpfError",
           "PRECISIONS"]

PRECISIONS = {"fp32": SPF_FP32, "bf16": SPF_BF16, "fp8": SPF_FP8}


def _dev_index(device) -> int:
    d = torch.device("cuda" if device is None else device)
    if d.type != "cuda":
        raise ValueError(f"device must be a CUDA device, got {d}")
    return torch.cuda.current_device() if d.index is None else d.index


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(dev: int):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _f32(t, name, dev, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    if t.device.type != "cuda" or t.device.index != dev:
        raise ValueError(f"{name} must live on cuda:{dev}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Plan:
    """NUFFT / merge plan for an N^3 model grid (Sec. II-A, II-C)."""

    def __init__(self, N: int, qmax: float = 1.0, eps: float = 1e-6, max_points: int = 0,
                 device=None):
        self.device = _dev_index(device)
        h = C.c_void_p()
        check(lib.spf_plan_create(C.byref(h), int(N), float(qmax), float(eps), int(max_points),
                                  self.device))
        self._h = h
        self.N, self.qmax, self.eps, self.max_points = int(N), float(qmax), float(eps), int(max_points)
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(lib.spf_plan_sizes(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        self.nf, self.nfT, self.PT, self.w = a.value, b.value, c.value, d.value

    @classmethod
    def view(cls, handle, N, qmax=1.0, eps=1e-6, device=None):
        """A non-owning Plan over a plan that another object (the M-TIP
        driver) created and destroys."""
        p = cls.__new__(cls)
        p.device = _dev_index(device)
        p._h = C.c_void_p(handle)
        p._owned = False
        p.N, p.qmax, p.eps, p.max_points = int(N), float(qmax), float(eps), 0
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(lib.spf_plan_sizes(p._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        p.nf, p.nfT, p.PT, p.w = a.value, b.value, c.value, d.value
        return p

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                lib.spf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self):
        check(lib.spf_plan_status(self._h))

    def _grid(self, t, name):
        return _f32(t, name, self.device, (self.N,) * 3)

    # -- Sec. II-A slicing and its adjoint ------------------------------------
    def slice_model(self, A, quats, q_lab, out=None):
        d = self.device
        self._grid(A, "A")
        _f32(quats, "quats", d)
        _f32(q_lab, "q_lab", d)
        M, P2 = quats.shape[0], q_lab.shape[0]
        if out is None:
            out = torch.empty((M, P2), dtype=torch.float32, device=A.device)
        _f32(out, "out", d, (M, P2))
        check(lib.spf_slice_model(self._h, _ptr(A), _ptr(quats), M, _ptr(q_lab), P2, _ptr(out),
                                  _stream(d)))
        return out

    def slice_adjoint(self, g, quats, q_lab, out=None, accumulate=False):
        d = self.device
        _f32(g, "g", d)
        _f32(quats, "quats", d)
        _f32(q_lab, "q_lab", d)
        M, P2 = quats.shape[0], q_lab.shape[0]
        if g.numel() != M * P2:
            raise ValueError("g must hold M * P2 values")
        if out is None:
            out = torch.empty((self.N,) * 3, dtype=torch.float32, device=g.device)
            accumulate = False
        self._grid(out, "out")
        check(lib.spf_slice_adjoint(self._h, _ptr(g), _ptr(quats), M, _ptr(q_lab), P2, _ptr(out),
                                    int(bool(accumulate)), _stream(d)))
        return out

    def nufft_type2(self, A, pts, out=None):
        d = self.device
        self._grid(A, "A")
        _f32(pts, "pts", d)
        n = pts.numel() // 3
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=A.device)
        check(lib.spf_nufft_type2(self._h, _ptr(A), _ptr(pts), n, _ptr(out), _stream(d)))
        return out

    def nufft_type1(self, v, pts, out=None, accumulate=False):
        d = self.device
        _f32(v, "v", d)
        _f32(pts, "pts", d)
        n = pts.numel() // 3
        if v.numel() != n:
            raise ValueError("v must hold one value per point")
        if out is None:
            out = torch.empty((self.N,) * 3, dtype=torch.float32, device=v.device)
            accumulate = False
        check(lib.spf_nufft_type1(self._h, _ptr(v), _ptr(pts), n, _ptr(out), int(bool(accumulate)),
                                  _stream(d)))
        return out

    # -- Sec. II-C merge: right-hand side, Toeplitz kernel, CG ----------------
    def merge_images(self, images, quats, q_lab, D=None, b_scale=1.0, rhs=None, kernel_hat=None,
                     accumulate=False, orient_idx=None, want_rhs=True, want_kernel=True):
        """Type-1 right-hand side and Toeplitz kernel of one image chunk.

        With orient_idx (int32, one per image) image i uses quats[orient_idx[i]];
        otherwise quats holds one row per image.
        """
        d = self.device
        _f32(quats, "quats", d)
        _f32(q_lab, "q_lab", d)
        P2 = q_lab.shape[0]
        if orient_idx is not None:
            if orient_idx.dtype != torch.int32 or not orient_idx.is_contiguous():
                raise TypeError("orient_idx must be a contiguous int32 tensor")
            n_img = orient_idx.shape[0]
        else:
            n_img = quats.shape[0]
        if want_rhs:
            _f32(images, "images", d, (n_img, P2))
        if D is not None:
            _f32(D, "D", d, (P2,))
        dev = quats.device
        if want_rhs and rhs is None:
            if accumulate:
                raise ValueError("accumulate needs an rhs tensor")
            rhs = torch.empty((self.N,) * 3, dtype=torch.float32, device=dev)
        if want_kernel and kernel_hat is None:
            if accumulate:
                raise ValueError("accumulate needs a kernel_hat tensor")
            kernel_hat = torch.empty((self.PT,) * 3, dtype=torch.float32, device=dev)
        if want_rhs:
            self._grid(rhs, "rhs")
        if want_kernel:
            _f32(kernel_hat, "kernel_hat", d, (self.PT,) * 3)
        check(lib.spf_merge_images(self._h, _ptr(images) if want_rhs else None, _ptr(quats),
                                   quats.shape[0], _ptr(orient_idx), n_img, _ptr(q_lab), P2, _ptr(D),
                                   float(b_scale), _ptr(rhs) if want_rhs else None,
                                   _ptr(kernel_hat) if want_kernel else None,
                                   int(bool(accumulate)), _stream(d)))
        return rhs, kernel_hat

    # -- deferred merge over many chunks (one transform of the summed grids) ---
    def merge_begin(self):
        check(lib.spf_merge_begin(self._h, _stream(self.device)))

    def merge_images_add(self, images, quats, q_lab, D=None, b_scale=1.0, orient_idx=None, want_rhs=True,
                         want_kernel=True):
        """Spread one image chunk onto the open merge (see merge_images)."""
        d = self.device
        _f32(quats, "quats", d)
        _f32(q_lab, "q_lab", d)
        P2 = q_lab.shape[0]
        if orient_idx is not None:
            if orient_idx.dtype != torch.int32 or not orient_idx.is_contiguous():
                raise TypeError("orient_idx must be a contiguous int32 tensor")
            n_img = orient_idx.shape[0]
        else:
            n_img = quats.shape[0]
        if want_rhs:
            _f32(images, "images", d, (n_img, P2))
        if D is not None:
            _f32(D, "D", d, (P2,))
        check(lib.spf_merge_images_add(self._h, _ptr(images) if want_rhs else None, _ptr(quats), quats.shape[0],
                                       _ptr(orient_idx), n_img, _ptr(q_lab), P2, _ptr(D), float(b_scale),
                                       int(bool(want_rhs)), int(bool(want_kernel)), _stream(d)))

    def merge_finish(self, rhs=None, kernel_hat=None, accumulate=False):
        """Transform the open merge's sums into rhs (N^3) and kernel_hat (P_T^3)."""
        d = self.device
        if rhs is not None:
            self._grid(rhs, "rhs")
        if kernel_hat is not None:
            _f32(kernel_hat, "kernel_hat", d, (self.PT,) * 3)
        check(lib.spf_merge_finish(self._h, _ptr(rhs), _ptr(kernel_hat), int(bool(accumulate)), _stream(d)))
        return rhs, kernel_hat

    def toeplitz_apply(self, kernel_hat, lam, x, out=None):
        d = self.device
        _f32(kernel_hat, "kernel_hat", d, (self.PT,) * 3)
        self._grid(x, "x")
        if out is None:
            out = torch.empty_like(x)
        check(lib.spf_toeplitz_apply(self._h, _ptr(kernel_hat), float(lam), _ptr(x), _ptr(out),
                                     _stream(d)))
        return out

    def cg_begin(self, kernel_hat, lam, rhs, x0, x=None, res=None):
        d = self.device
        _f32(kernel_hat, "kernel_hat", d, (self.PT,) * 3)
        self._grid(rhs, "rhs")
        self._grid(x0, "x0")
        if x is None:
            x = torch.empty_like(x0)
        self._grid(x, "x")
        check(lib.spf_cg_begin(self._h, _ptr(kernel_hat), float(lam), _ptr(rhs), _ptr(x0), _ptr(x),
                               _ptr(res), _stream(d)))
        return x

    def cg_merge_step(self, kernel_hat, lam, x, res=None):
        d = self.device
        _f32(kernel_hat, "kernel_hat", d, (self.PT,) * 3)
        self._grid(x, "x")
        if res is not None and (res.dtype != torch.float64 or res.numel() < 1):
            raise TypeError("res must be a float64 device tensor")
        check(lib.spf_cg_merge_step(self._h, _ptr(kernel_hat), float(lam), _ptr(x), _ptr(res),
                                    _stream(d)))
        return x

    def cg_solve(self, kernel_hat, lam, rhs, x0, iters, x=None, res_hist=None):
        """x after `iters` CG steps from x0; res_hist (float64, iters+1) gets |r_k|."""
        x = self.cg_begin(kernel_hat, lam, rhs, x0, x=x,
                          res=None if res_hist is None else res_hist[0:1])
        for k in range(iters):
            self.cg_merge_step(kernel_hat, lam, x,
                               res=None if res_hist is None else res_hist[k + 1:k + 2])
        return x


class PointSet:
    """Rotated detector points of a fixed orientation set, sorted once (Sec. II-A:
    the model images live on a predetermined orientation set)."""

    SLICE_ONLY = 1   # SPF_POINTS_SLICE_ONLY

    def __init__(self, plan: Plan, quats, q_lab, slice_only=False):
        """slice_only: sort for slicing alone (4 bytes per point; no merge)."""
        d = plan.device
        _f32(quats, "quats", d)
        _f32(q_lab, "q_lab", d)
        self.plan = plan
        self.M, self.P2 = quats.shape[0], q_lab.shape[0]
        h = C.c_void_p()
        check(lib.spf_points_create(C.byref(h), plan._h, _ptr(quats), self.M, _ptr(q_lab), self.P2,
                                    self.SLICE_ONLY if slice_only else 0, _stream(d)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.spf_points_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def slice(self, A, out=None):
        """Model images (M, P2) of model A at the set's orientations."""
        p, d = self.plan, self.plan.device
        p._grid(A, "A")
        if out is None:
            out = torch.empty((self.M, self.P2), dtype=torch.float32, device=A.device)
        _f32(out, "out", d, (self.M, self.P2))
        check(lib.spf_slice_points(p._h, self._h, _ptr(A), _ptr(out), _stream(d)))
        return out

    def merge_add(self, images, orient_idx, orient_offset=0, D=None, b_scale=1.0, want_rhs=True,
                  want_kernel=True):
        """Class sums of this set's orientations spread onto the plan's open
        merge (Plan.merge_begin ... Plan.merge_finish)."""
        p, d = self.plan, self.plan.device
        _f32(images, "images", d)
        if orient_idx.dtype != torch.int32 or not orient_idx.is_contiguous():
            raise TypeError("orient_idx must be a contiguous int32 tensor")
        n_img = images.shape[0]
        if images.dim() != 2 or images.shape[1] != self.P2 or orient_idx.shape[0] != n_img:
            raise ValueError("images must be (n, P2) with one orient_idx per image")
        if D is not None:
            _f32(D, "D", d, (self.P2,))
        check(lib.spf_merge_points_add(p._h, self._h, _ptr(images), _ptr(orient_idx), n_img, int(orient_offset),
                                       _ptr(D), float(b_scale), int(bool(want_rhs)), int(bool(want_kernel)),
                                       _stream(d)))

    def merge(self, images, orient_idx, orient_offset=0, D=None, b_scale=1.0, rhs=None, kernel_hat=None,
              accumulate=False, want_rhs=True, want_kernel=True):
        """Sec. II-C right-hand side and Toeplitz kernel from class sums of the
        images whose orient_idx lies in [orient_offset, orient_offset + M)."""
        p, d = self.plan, self.plan.device
        _f32(images, "images", d)
        if orient_idx.dtype != torch.int32 or not orient_idx.is_contiguous():
            raise TypeError("orient_idx must be a contiguous int32 tensor")
        n_img = images.shape[0]
        if images.dim() != 2 or images.shape[1] != self.P2 or orient_idx.shape[0] != n_img:
            raise ValueError("images must be (n, P2) with one orient_idx per image")
        if D is not None:
            _f32(D, "D", d, (self.P2,))
        if want_rhs and rhs is None:
            if accumulate:
                raise ValueError("accumulate needs an rhs tensor")
            rhs = torch.empty((p.N,) * 3, dtype=torch.float32, device=images.device)
        if want_kernel and kernel_hat is None:
            if accumulate:
                raise ValueError("accumulate needs a kernel_hat tensor")
            kernel_hat = torch.empty((p.PT,) * 3, dtype=torch.float32, device=images.device)
        check(lib.spf_merge_points(p._h, self._h, _ptr(images), _ptr(orient_idx), n_img, int(orient_offset),
                                   _ptr(D), float(b_scale), _ptr(rhs) if want_rhs else None,
                                   _ptr(kernel_hat) if want_kernel else None, int(bool(accumulate)),
                                   _stream(d)))
        return rhs, kernel_hat


class Matcher:
    """Orientation matcher (Sec. II-B) with a streaming top-k across chunks."""

    def __init__(self, max_images: int, max_orient_chunk: int, P2: int, precision="bf16",
                 topk: int = 8, device=None):
        self.device = _dev_index(device)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = C.c_void_p()
        check(lib.spf_matcher_create(C.byref(h), int(max_images), int(max_orient_chunk), int(P2),
                                     self.precision, int(topk), self.device))
        self._h = h
        self.P2, self.topk = int(P2), int(topk)
        self.max_images, self.max_orient = int(max_images), int(max_orient_chunk)
        self._images = None
        self.n_img = 0

    @classmethod
    def view(cls, handle, max_images, max_orient_chunk, P2, precision="bf16", topk=8, device=None):
        """A non-owning Matcher over a matcher the M-TIP driver owns."""
        m = cls.__new__(cls)
        m.device = _dev_index(device)
        m.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        m._h = C.c_void_p(handle)
        m._owned = False
        m.P2, m.topk = int(P2), int(topk)
        m.max_images, m.max_orient = int(max_images), int(max_orient_chunk)
        m._images = None
        m.n_img = 0
        return m

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                lib.spf_matcher_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self):
        check(lib.spf_matcher_status(self._h))

    def set_mask(self, D=None):
        """Pixel weights D (P2,) for the distance (0 excludes a pixel); None clears."""
        if D is not None:
            _f32(D, "D", self.device, (self.P2,))
        self._mask = D
        check(lib.spf_matcher_set_mask(self._h, _ptr(D), _stream(self.device)))

    def set_schedule(self, schedule="auto"):
        """Tile schedule of the tensor-core cross term: "auto", "contiguous" or "grid"."""
        check(lib.spf_matcher_set_schedule(self._h, {"auto": 0, "contiguous": 1, "grid": 2}[schedule]))

    def set_rerank(self, deferred=False):
        """Re-rank per add_slices call (False) or once, at results, over the
        running approximate top-8 of all chunks (True: every chunk's slices must
        stay valid until results)."""
        check(lib.spf_matcher_set_rerank(self._h, int(bool(deferred))))

    def set_images(self, images, img_scale=1.0):
        """FP32 images, or (BF16 / FP8 matchers) 16-bit photon counts, which
        the quantisation and the FP32 re-rank read directly."""
        counts = images.dtype in COUNT_DTYPES
        if counts:
            if images.device.type != "cuda" or images.device.index != self.device or not images.is_contiguous():
                raise ValueError("images must be a contiguous tensor on the matcher's device")
        else:
            _f32(images, "images", self.device)
        if images.dim() != 2 or images.shape[1] != self.P2:
            raise ValueError(f"images must be (n, {self.P2})")
        self._images = images          # the C side keeps this pointer
        self.n_img = images.shape[0]
        fn = lib.spf_matcher_set_images_u16 if counts else lib.spf_matcher_set_images
        check(fn(self._h, _ptr(images), self.n_img, float(img_scale), _stream(self.device)))

    def add_slices(self, slices, orient_offset=0):
        _f32(slices, "slices", self.device)
        if slices.dim() != 2 or slices.shape[1] != self.P2:
            raise ValueError(f"slices must be (m, {self.P2})")
        check(lib.spf_matcher_add_slices(self._h, _ptr(slices), slices.shape[0], int(orient_offset),
                                         _stream(self.device)))

    def results(self, with_topk=False):
        n, dev = self.n_img, torch.device("cuda", self.device)
        best = torch.empty(n, dtype=torch.int32, device=dev)
        d1 = torch.empty(n, dtype=torch.float32, device=dev)
        d2 = torch.empty(n, dtype=torch.float32, device=dev)
        ti = td = None
        if with_topk:
            ti = torch.empty((n, self.topk), dtype=torch.int32, device=dev)
            td = torch.empty((n, self.topk), dtype=torch.float32, device=dev)
        check(lib.spf_matcher_results(self._h, _ptr(best), _ptr(d1), _ptr(d2), _ptr(ti), _ptr(td),
                                      _stream(self.device)))
        out = {"best": best, "d1": d1, "d2": d2}
        if with_topk:
            out["topk_idx"], out["topk_d"] = ti, td
        return out

    def match(self, images, slices, img_scale=1.0):
        """One-shot match_orientations: (best index, best distance, second distance)."""
        _f32(images, "images", self.device)
        _f32(slices, "slices", self.device)
        n = images.shape[0]
        dev = images.device
        best = torch.empty(n, dtype=torch.int32, device=dev)
        d1 = torch.empty(n, dtype=torch.float32, device=dev)
        d2 = torch.empty(n, dtype=torch.float32, device=dev)
        self._images = images
        self.n_img = n
        check(lib.spf_match_orientations(self._h, _ptr(images), n, float(img_scale), _ptr(slices),
                                         slices.shape[0], _ptr(best), _ptr(d1), _ptr(d2),
                                         _stream(self.device)))
        return best, d1, d2


class SliceModel(torch.autograd.Function):
    """slices = Re type-2 NUFFT of A at rotated detector points (Sec. II-A).

    backward is the hand-written adjoint (type-1 spread, Sec. II-C). Nothing
    but the orientations and q-points is saved: the backward never needs the
    slices, so memory holds only what the caller keeps.
    """

    @staticmethod
    def forward(ctx, A, quats, q_lab, plan):
        ctx.plan = plan
        ctx.save_for_backward(quats, q_lab)
        return plan.slice_model(A.contiguous(), quats, q_lab)

    @staticmethod
    def backward(ctx, g):
        quats, q_lab = ctx.saved_tensors
        gA = ctx.plan.slice_adjoint(g.contiguous(), quats, q_lab)
        return gA, None, None, None


def slice_model(A, quats, q_lab, plan: Plan):
    return SliceModel.apply(A, quats, q_lab, plan)


COUNT_DTYPES = (torch.int16, torch.uint16) if hasattr(torch, "uint16") else (torch.int16,)


def counts_to_f32(counts, out=None):
    """FP32 copy of 16-bit photon-count images on their device. An int16
    tensor is read as the unsigned 16-bit pattern (0 .. 65535), so counts
    above 32767 survive a round trip through int16."""
    if not isinstance(counts, torch.Tensor) or counts.dtype not in COUNT_DTYPES:
        raise TypeError("counts must be an int16 or uint16 torch.Tensor")
    if counts.device.type != "cuda" or not counts.is_contiguous():
        raise ValueError("counts must be a contiguous CUDA tensor")
    d = counts.device.index
    if out is None:
        out = torch.empty(counts.shape, dtype=torch.float32, device=counts.device)
    _f32(out, "out", d, counts.shape)
    check(lib.spf_counts_to_f32(_ptr(counts), counts.numel(), _ptr(out), _stream(d)))
    return out
