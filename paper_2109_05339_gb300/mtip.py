"""One slice -> match -> merge -> CG iteration of M-TIP on one GPU (Fig. 3
without phasing): a thin binding of the library's native driver
(spf_mtip_* in include/spf.h), which orchestrates the kernels.

The reference orientations are fixed across iterations (Sec. II-A), so the
driver takes the orientation set once: it renumbers it along a Morton curve of
the quaternions and sorts the rotated points of every orientation chunk once
(kept, 16 bytes per orientation x pixel) or, beyond the memory budget (e.g.
the paper's 1.2 million orientations of 128 x 128 pixels, 315 GB), re-sorts
them per chunk for slicing on every iteration and merges image chunks at their
matched orientations. The binding re-sends the set when the caller passes
other tensors, or the same tensors written in place through torch (their
version counter moved); the driver keeps its own copies.

1. Slicing (Sec. II-A) and matching (Sec. II-B), streamed in orientation
   chunks; the running top-k survives across chunks.
2. Merging (Sec. II-C): every chunk is spread onto the plan's fine grids,
   transformed once into the right-hand side and the Toeplitz kernel
   (linearity, the paper's per-node type-1 sums and reduction).
3. ``cg_iters`` conjugate-gradient steps on Eq. 2 from x0 = current model,
   lambda = lam_rel * sum of the weights D over all merged pixels.

With a process group the images are one shard: the right-hand side and the
kernel are summed over the ranks between merge and solve, and lambda takes
the global image count.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import SPF_IMAGES_F32, SPF_IMAGES_U16, SPF_UPLOAD_COPY, SPF_UPLOAD_SM, MtipConfig, check, lib
from .api import COUNT_DTYPES, PRECISIONS, Matcher, Plan, _dev_index, _f32, _ptr, _stream
from .dist import allreduce_sum_, global_count


class _DevArray:
    # a device buffer of the library seen by torch without a copy
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _device_view(ptr, shape, typestr, device):
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device=torch.device("cuda", device))


def morton_order(quats_host):
    """The driver's renumbering: permutation sorting unit quaternions (w, x, y,
    z) by the Morton code of (x, y, z) quantised to 10 bits per axis."""
    q = np.ascontiguousarray(np.asarray(quats_host, dtype=np.float32))
    M = q.shape[0]
    out = np.empty(M, dtype=np.int32)
    check(lib.spf_morton_order(q.ctypes.data_as(C.c_void_p), M, out.ctypes.data_as(C.c_void_p)))
    return out.astype(np.int64)


def _tensor_key(t):
    """Identity of a tensor's contents as far as torch can tell without reading
    them: storage, shape, and the version counter that every in-place write
    through torch increments."""
    return (t.data_ptr(), tuple(t.shape), t._version)


_POINT_MODES = {None: -1, True: 1, False: 0, "slices": 2}


class MTIP:
    def __init__(self, N, qmax, P2, n_img, n_orient, orient_chunk=None, img_chunk=None,
                 eps=1e-6, precision="bf16", topk=8, device=None, cache_points=None,
                 point_budget_bytes=None, process_group=None, host_images=None, keep_slices=None):
        """cache_points: keep every chunk's sorted points (True), keep only
        their sort for slicing and merge image chunks ("slices"), re-sort per
        chunk on every call (False), or decide from point_budget_bytes (None:
        the first of these that fits; default budget: half of the device's free
        memory). process_group: the images are one shard
        of a torch.distributed group. host_images: None, "f32" or "u16" --
        the image type of iteration_host (allocates its two device slots).
        keep_slices: keep every chunk's slices and re-rank once per iteration
        (True), re-rank per chunk (False), or decide from free memory (None)."""
        if cache_points not in _POINT_MODES:
            raise ValueError(f"cache_points must be None, True, False or 'slices', not {cache_points!r}")
        self.group = process_group
        self._n_total = {}
        dev = _dev_index(device)
        cfg = MtipConfig(N=int(N), qmax=float(qmax), eps=float(eps), P2=int(P2), max_images=int(n_img),
                         n_orient=int(n_orient), orient_chunk=int(orient_chunk or 0),
                         img_chunk=int(img_chunk or 0),
                         precision=PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                         topk=int(topk), cache_points=_POINT_MODES[cache_points],
                         point_budget_bytes=int(point_budget_bytes or 0),
                         host_image_type={None: -1, "f32": SPF_IMAGES_F32, "u16": SPF_IMAGES_U16}[host_images],
                         device=dev, keep_slices=-1 if keep_slices is None else int(bool(keep_slices)))
        h = C.c_void_p()
        check(lib.spf_mtip_create(C.byref(h), C.byref(cfg)))
        self._h = h
        cp, oc, ic, ks = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(lib.spf_mtip_info(h, C.byref(cp), C.byref(oc), C.byref(ic), C.byref(ks)))
        self.cache_points, self.orient_chunk, self.img_chunk = cp.value == 1, oc.value, ic.value
        self.point_mode = {1: "cached", 2: "slice sets kept", 0: "streamed"}[cp.value]
        self.keep_slices = bool(ks.value)
        self.device = dev
        self.N, self.P2, self.n_img, self.n_orient, self.topk = int(N), int(P2), int(n_img), int(n_orient), int(topk)
        self.host_images = host_images
        self.plan = Plan.view(lib.spf_mtip_plan(h), N, qmax, eps, device=dev)
        self.matcher = Matcher.view(lib.spf_mtip_matcher(h), n_img, self.orient_chunk, P2, precision, topk,
                                    device=dev)
        d = torch.device("cuda", dev)
        self.rhs = torch.empty((N,) * 3, dtype=torch.float32, device=d)
        self.khat = torch.empty((self.plan.PT,) * 3, dtype=torch.float32, device=d)
        self.x = torch.empty((N,) * 3, dtype=torch.float32, device=d)
        self._best = torch.empty(n_img, dtype=torch.int32, device=d)
        self._key = None
        self._orient = None
        self._mask = None

    # -- configuration --------------------------------------------------------
    def set_orientations(self, quats, q_lab, force=False):
        """Give the driver the orientation set and detector (sorted once);
        repeated calls with unchanged tensors do nothing unless force is set."""
        _f32(quats, "quats", self.device, (self.n_orient, 4))
        _f32(q_lab, "q_lab", self.device, (self.P2, 3))
        key = (_tensor_key(quats), _tensor_key(q_lab))
        if key == self._key and not force:
            return
        self._key = None
        check(lib.spf_mtip_set_orientations(self._h, _ptr(quats), _ptr(q_lab), _stream(self.device)))
        self._key = key
        self._orient = (quats, q_lab)

    def set_mask(self, D):
        """Pixel weights D (P2,) for matching, merging and lambda; None: ones."""
        key = None if D is None else _tensor_key(D)
        if key == self._mask:
            return
        if D is not None:
            _f32(D, "D", self.device, (self.P2,))
        self._D = D                       # the driver keeps the pointer
        check(lib.spf_mtip_set_mask(self._h, _ptr(D), _stream(self.device)))
        self._mask = key

    def _images(self, images):
        if images.dtype in COUNT_DTYPES:
            t = SPF_IMAGES_U16
        elif images.dtype == torch.float32:
            t = SPF_IMAGES_F32
        else:
            raise TypeError("images must be float32, or 16-bit photon counts (int16 read as unsigned, uint16)")
        if images.device.type != "cuda" or images.device.index != self.device or not images.is_contiguous():
            raise ValueError(f"images must be contiguous on cuda:{self.device}")
        if images.dim() != 2 or images.shape[1] != self.P2 or not 1 <= images.shape[0] <= self.n_img:
            raise ValueError(f"images must be (n, {self.P2}) with 1 <= n <= {self.n_img}")
        return t

    # -- the three steps --------------------------------------------------------
    def match(self, A, quats, q_lab, images, img_scale, with_topk=False):
        """Per image the best orientation (caller's numbering), best and
        second distances, optionally the re-ranked top-k."""
        self.set_orientations(quats, q_lab)
        self.plan._grid(A, "A")
        t = self._images(images)
        n, d = images.shape[0], images.device
        best = torch.empty(n, dtype=torch.int32, device=d)
        d1 = torch.empty(n, dtype=torch.float32, device=d)
        d2 = torch.empty(n, dtype=torch.float32, device=d)
        ti = td = None
        if with_topk:
            ti = torch.empty((n, self.topk), dtype=torch.int32, device=d)
            td = torch.empty((n, self.topk), dtype=torch.float32, device=d)
        check(lib.spf_mtip_match(self._h, _ptr(A), _ptr(images), t, n, C.c_float(img_scale), _ptr(best), _ptr(d1),
                                 _ptr(d2), _ptr(ti), _ptr(td), _stream(self.device)))
        out = {"best": best, "d1": d1, "d2": d2}
        if with_topk:
            out["topk_idx"], out["topk_d"] = ti, td
        return out

    def merge(self, images, quats, q_lab, best, img_scale, rhs=None, kernel_hat=None):
        """Right-hand side and Toeplitz-kernel spectrum of the images at
        orientations best (caller's numbering, int32)."""
        self.set_orientations(quats, q_lab)
        t = self._images(images)
        if best.dtype != torch.int32 or not best.is_contiguous() or best.shape != (images.shape[0],):
            raise ValueError("best must be a contiguous int32 tensor, one per image")
        rhs = self.rhs if rhs is None else self.plan._grid(rhs, "rhs")
        kernel_hat = self.khat if kernel_hat is None else _f32(kernel_hat, "kernel_hat", self.device,
                                                               (self.plan.PT,) * 3)
        check(lib.spf_mtip_merge(self._h, _ptr(images), t, images.shape[0], C.c_float(img_scale), _ptr(best),
                                 _ptr(rhs), _ptr(kernel_hat), _stream(self.device)))
        return rhs, kernel_hat

    def solve_system(self, rhs, kernel_hat, x0, lam_rel, n_img_total, cg_iters, x=None, res_hist=None):
        """CG on Eq. 2 from x0; returns (x, lambda)."""
        x = self.x if x is None else self.plan._grid(x, "x")
        if res_hist is not None and (res_hist.dtype != torch.float64 or res_hist.numel() < cg_iters + 1):
            raise ValueError("res_hist must be a float64 device tensor of cg_iters + 1 values")
        lam = C.c_double()
        check(lib.spf_mtip_solve(self._h, _ptr(rhs), _ptr(kernel_hat), _ptr(self.plan._grid(x0, "x0")),
                                 float(lam_rel), int(n_img_total), int(cg_iters), _ptr(x), C.byref(lam),
                                 _ptr(res_hist), _stream(self.device)))
        return x, lam.value

    def _global_count(self, n):
        if self.group is None:
            return n
        if n not in self._n_total:
            self._n_total[n] = global_count(n, torch.device("cuda", self.device), self.group)
        return self._n_total[n]

    def solve(self, A, quats, q_lab, images, img_scale, best, cg_iters, lam_rel=1e-3, D=None, res_hist=None):
        """The merge and solve half of an iteration at given orientations:
        image i merged at orientation best[i] (caller's numbering), then
        cg_iters CG steps from x0 = A. Returns (x, lambda)."""
        self.set_mask(D)
        rhs, kh = self.merge(images, quats, q_lab, best, img_scale)
        if self.group is not None:
            allreduce_sum_([rhs, kh], self.group)
        return self.solve_system(rhs, kh, A, lam_rel, self._global_count(images.shape[0]), cg_iters,
                                 res_hist=res_hist)

    def iteration(self, A, quats, q_lab, images, img_scale, cg_iters, lam_rel=1e-3, D=None, res_hist=None):
        """Returns (match results, merged model x, lambda). images: FP32, or
        16-bit photon counts (int16 read as unsigned, or uint16)."""
        self.set_mask(D)
        if self.group is None and res_hist is None:
            self.set_orientations(quats, q_lab)
            self.plan._grid(A, "A")
            t = self._images(images)
            n = images.shape[0]
            best = self._best[:n]
            lam = C.c_double()
            check(lib.spf_mtip_iteration(self._h, _ptr(A), _ptr(images), t, n, C.c_float(img_scale), int(cg_iters),
                                         float(lam_rel), _ptr(best), _ptr(self.x), C.byref(lam),
                                         _stream(self.device)))
            return {"best": best}, self.x, lam.value
        res = self.match(A, quats, q_lab, images, img_scale)
        x, lam = self.solve(A, quats, q_lab, images, img_scale, res["best"], cg_iters, lam_rel, D, res_hist)
        return res, x, lam

    def iteration_host(self, A_host, images_host, img_scale, cg_iters, lam_rel=1e-3, best_out=None, x_out=None):
        """The iteration from host buffers (page-locked for overlap): the
        inputs are copied on the driver's copy stream while the previous call
        computes; best_out (int32, n) and x_out (float32, N^3) are host tensors
        written when the current stream reaches the end of this call's work.
        Returns (best_out, x_out, lambda)."""
        if self.host_images is None:
            raise ValueError("construct the driver with host_images='f32' or 'u16' for host-buffer iterations")
        want = torch.float32 if self.host_images == "f32" else None
        if A_host.device.type != "cpu" or images_host.device.type != "cpu":
            raise ValueError("iteration_host takes host tensors")
        if (want is not None and images_host.dtype != want) or \
                (want is None and images_host.dtype not in COUNT_DTYPES):
            raise TypeError(f"images_host must be {self.host_images}")
        if A_host.dtype != torch.float32 or tuple(A_host.shape) != (self.N,) * 3 or not A_host.is_contiguous():
            raise ValueError(f"A_host must be a contiguous float32 ({self.N},)*3 host tensor")
        if not images_host.is_contiguous() or images_host.dim() != 2 or images_host.shape[1] != self.P2:
            raise ValueError(f"images_host must be a contiguous (n, {self.P2}) host tensor")
        n = images_host.shape[0]
        if best_out is None:
            best_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
        if x_out is None:
            x_out = torch.empty((self.N,) * 3, dtype=torch.float32, pin_memory=True)
        t = SPF_IMAGES_F32 if self.host_images == "f32" else SPF_IMAGES_U16
        if self.group is not None:
            return self._iteration_host_group(A_host, images_host, t, img_scale, cg_iters, lam_rel, best_out, x_out)
        lam = C.c_double()
        check(lib.spf_mtip_iteration_host(self._h, _ptr(A_host), _ptr(images_host), t, n, C.c_float(img_scale),
                                          int(cg_iters), float(lam_rel), _ptr(best_out), _ptr(x_out),
                                          C.byref(lam), _stream(self.device)))
        return best_out, x_out, lam.value

    def set_upload(self, mode):
        """How iteration_host moves the images: 'sm' (default: a kernel reads
        the page-locked host buffer; falls back to the copy engines for
        buffers that are not one mapped page-locked range) or 'copy' (copy
        engines only)."""
        check(lib.spf_mtip_set_upload(self._h, {"copy": SPF_UPLOAD_COPY, "sm": SPF_UPLOAD_SM}[mode]))

    def last_upload_ms(self):
        """Device time of the latest image upload of iteration_host (-1 before
        the first); waits for it."""
        ms = C.c_float()
        check(lib.spf_mtip_last_upload_ms(self._h, C.byref(ms)))
        return ms.value

    def _iteration_host_group(self, A_host, images_host, t, img_scale, cg_iters, lam_rel, best_out, x_out):
        # image-sharded: the library uploads into its slot, the steps run with
        # the merge sums reduced over the group between merge and solve
        if getattr(self, "_orient", None) is None:
            raise RuntimeError("set_orientations first")
        n = images_host.shape[0]
        a_dev, i_dev = C.c_void_p(), C.c_void_p()
        st = _stream(self.device)
        check(lib.spf_mtip_upload_host(self._h, _ptr(A_host), _ptr(images_host), t, n, C.byref(a_dev),
                                       C.byref(i_dev), st))
        try:
            A = _device_view(a_dev.value, (self.N,) * 3, "<f4", self.device)
            imgs = _device_view(i_dev.value, (n, self.P2), "<f4" if t == SPF_IMAGES_F32 else "<i2", self.device)
            q, ql = self._orient
            res = self.match(A, q, ql, imgs, img_scale)
            x, lam = self.solve(A, q, ql, imgs, img_scale, res["best"], cg_iters, lam_rel)
            best_out.copy_(res["best"], non_blocking=True)
            x_out.copy_(x, non_blocking=True)
        finally:
            check(lib.spf_mtip_release_upload(self._h, st))
        return best_out, x_out, lam

    def status(self):
        check(lib.spf_mtip_status(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib.spf_mtip_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
