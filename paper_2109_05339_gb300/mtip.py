"""One slice -> match -> merge -> CG iteration of M-TIP on one GPU (Fig. 3
without phasing), as a sequence of C-ABI calls.

The reference orientations are fixed across iterations (Sec. II-A), so their
rotated detector points are sorted once per orientation chunk (PointSet) and
reused by every iteration's slicing and merge. A point set costs 16 bytes per
(orientation, pixel); when the whole set would not fit the memory budget
(e.g. the paper's 1.2 million orientations of 128 x 128 pixels, 315 GB) the
driver streams instead: each chunk's points are sorted (for slicing only,
4 bytes per point), sliced and matched, then released, and the merge spreads
the images at their matched orientations (image chunks accumulate).

The driver numbers the reference orientations along a space-filling (Morton)
curve of their quaternions, so that orientations close in index are close on
SO(3): images re-ranked together then share candidate model images, which
stay in L2. Indices returned to the caller are in the caller's numbering
(an exact distance tie resolves to the lower index in the driver's numbering).

1. Slicing (Sec. II-A) and matching (Sec. II-B), streamed in orientation
   chunks: each chunk of model images is sliced into one reusable buffer and
   matched against every image; the running top-k survives across chunks, so
   no more than one chunk of slices is resident.
2. Merging (Sec. II-C): images are summed per matched orientation (class
   sums) and the sums and class counts are spread at the fixed points; chunks
   accumulate (linearity, the paper's per-node type-1 sums and reduction).
3. ``cg_iters`` conjugate-gradient steps on Eq. 2 from x0 = current model,
   lambda = lam_rel * sum of the weights D over all merged pixels.
"""
from __future__ import annotations

import numpy as np
import torch

from .api import COUNT_DTYPES, Matcher, Plan, PointSet, counts_to_f32
from .dist import allreduce_sum_, global_count


def morton_order(quats_host):
    """Permutation sorting unit quaternions (w, x, y, z; w >= 0) by the Morton
    code of (x, y, z) quantised to 10 bits per axis."""
    q = np.asarray(quats_host, dtype=np.float64)
    c = np.clip(((q[:, 1:4] + 1.0) * 0.5 * 1023.0).round(), 0, 1023).astype(np.uint64)
    key = np.zeros(q.shape[0], dtype=np.uint64)
    for bit in range(10):
        for a in range(3):
            key |= ((c[:, a] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(3 * bit + a)
    return np.argsort(key, kind="stable")


POINT_SET_BYTES = 16   # per (orientation, pixel): two sort orders, inverse order, class sum


class MTIP:
    def __init__(self, N, qmax, P2, n_img, n_orient, orient_chunk=None, img_chunk=None,
                 eps=1e-6, precision="bf16", topk=8, device=None, cache_points=None,
                 point_budget_bytes=None, process_group=None):
        """cache_points: keep every chunk's sorted points across iterations
        (True), stream them (False), or decide from point_budget_bytes (None;
        default budget: half of the device's free memory at construction).
        process_group: the images are one shard of a torch.distributed group;
        the merge's sums and the image count are added over its ranks."""
        self.group = process_group
        self._n_total = {}   # local image count -> count over the group
        self.orient_chunk = min(n_orient, orient_chunk or n_orient)
        if device is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        else:
            dev = device if isinstance(device, torch.device) else torch.device("cuda", int(device))
        if cache_points is None:
            if point_budget_bytes is None:
                free, _ = torch.cuda.mem_get_info(dev)
                point_budget_bytes = free // 2
            cache_points = POINT_SET_BYTES * n_orient * P2 <= point_budget_bytes
        self.cache_points = bool(cache_points)
        # the plan's own sort buffers serve per-call slicing of one orientation
        # chunk and, when streaming, the merge of one image chunk (< 2^31 points)
        self.img_chunk = min(n_img, img_chunk or n_img, (2 ** 31 - 1) // P2)
        max_pts = self.orient_chunk * P2
        if not self.cache_points:
            max_pts = max(max_pts, self.img_chunk * P2)
        self.plan = Plan(N, qmax, eps, max_points=max_pts, device=device)
        self.device = self.plan.device
        self.matcher = Matcher(n_img, self.orient_chunk, P2, precision, topk, device=self.device)
        dev = torch.device("cuda", self.device)
        self.slices = torch.empty((self.orient_chunk, P2), dtype=torch.float32, device=dev)
        self.rhs = torch.empty((N,) * 3, dtype=torch.float32, device=dev)
        self.khat = torch.empty((self.plan.PT,) * 3, dtype=torch.float32, device=dev)
        self.x = torch.empty((N,) * 3, dtype=torch.float32, device=dev)
        self.N, self.P2, self.n_img, self.n_orient = N, P2, n_img, n_orient
        self.sets = None
        self._key = None
        self._okey = None
        self.order = None   # sorted index -> caller's orientation index (int64, device)
        self.quats_sorted = None
        self._img32 = None   # FP32 images converted from 16-bit counts

    def _order_orientations(self, quats):
        """Renumber the orientation set along the Morton curve (once per set)."""
        okey = (quats.data_ptr(), tuple(quats.shape))
        if self._okey == okey:
            return
        order = morton_order(quats.detach().cpu().numpy())
        self.order = torch.as_tensor(order, dtype=torch.int64, device=quats.device)
        self.quats_sorted = quats.index_select(0, self.order).contiguous()
        self._okey = okey

    def set_orientations(self, quats, q_lab):
        """Sort the points of every orientation chunk once (reused by later calls)."""
        self._order_orientations(quats)
        key = (quats.data_ptr(), tuple(quats.shape), q_lab.data_ptr(), tuple(q_lab.shape))
        if self._key == key:
            return
        if self.sets:
            for _, s in self.sets:
                s.close()
        self.sets = []
        qs = self.quats_sorted
        M = qs.shape[0]
        for c0 in range(0, M, self.orient_chunk):
            c1 = min(M, c0 + self.orient_chunk)
            self.sets.append((c0, PointSet(self.plan, qs[c0:c1].contiguous(), q_lab)))
        self._key = key

    def _to_caller(self, res):
        """Match results with orientation indices in the caller's numbering;
        the sorted-numbering best index is kept under 'best_sorted'."""
        out = dict(res)
        out["best_sorted"] = res["best"]
        out["best"] = self.order.index_select(0, res["best"].long()).to(torch.int32)
        if "topk_idx" in res:
            ti = res["topk_idx"].long()
            out["topk_idx"] = self.order.index_select(0, ti.clamp(min=0).reshape(-1)).reshape(ti.shape) \
                .to(torch.int32).masked_fill(ti < 0, -1)
        return out

    def match(self, A, quats, q_lab, images, img_scale, with_topk=False):
        """Match every image against the orientation set; indices in the
        caller's numbering ('best_sorted': the driver's own numbering)."""
        m = self.matcher
        m.set_images(images, img_scale)
        if self.cache_points:
            self.set_orientations(quats, q_lab)
            for c0, ps in self.sets:
                sl = self.slices[: ps.M]
                ps.slice(A, out=sl)
                m.add_slices(sl, orient_offset=c0)
            return self._to_caller(m.results(with_topk))
        self._order_orientations(quats)
        qs = self.quats_sorted
        M = qs.shape[0]
        for c0 in range(0, M, self.orient_chunk):
            c1 = min(M, c0 + self.orient_chunk)
            ps = PointSet(self.plan, qs[c0:c1].contiguous(), q_lab, slice_only=True)
            sl = self.slices[: c1 - c0]
            ps.slice(A, out=sl)
            m.add_slices(sl, orient_offset=c0)
            ps.close()
        return self._to_caller(m.results(with_topk))

    def merge(self, images, quats, best_sorted, q_lab, img_scale, D=None):
        """Merge at the matched orientations, given in the driver's numbering
        (the 'best_sorted' of match)."""
        if self.cache_points:
            self.set_orientations(quats, q_lab)
            for k, (c0, ps) in enumerate(self.sets):
                ps.merge(images, best_sorted, orient_offset=c0, D=D, b_scale=img_scale, rhs=self.rhs,
                         kernel_hat=self.khat, accumulate=k > 0)
            return self.rhs, self.khat
        self._order_orientations(quats)
        n = images.shape[0]
        for i0 in range(0, n, self.img_chunk):
            i1 = min(n, i0 + self.img_chunk)
            self.plan.merge_images(images[i0:i1], self.quats_sorted, q_lab, D=D, b_scale=img_scale,
                                   rhs=self.rhs, kernel_hat=self.khat, accumulate=i0 > 0,
                                   orient_idx=best_sorted[i0:i1].contiguous())
        return self.rhs, self.khat

    def _images_f32(self, images):
        """The images as FP32: 16-bit photon counts are converted on the
        device into a buffer kept by the driver."""
        if images.dtype not in COUNT_DTYPES:
            return images
        if self._img32 is None or self._img32.shape != images.shape or self._img32.device != images.device:
            self._img32 = torch.empty(images.shape, dtype=torch.float32, device=images.device)
        return counts_to_f32(images, out=self._img32)

    def iteration(self, A, quats, q_lab, images, img_scale, cg_iters, lam_rel=1e-3, D=None,
                  d_sum=None, res_hist=None):
        """Returns (match results, merged model x, lambda); d_sum = sum of D over one image.
        images: FP32, or 16-bit photon counts (int16 read as unsigned, or uint16)."""
        images = self._images_f32(images)
        res = self.match(A, quats, q_lab, images, img_scale)
        self.merge(images, quats, res["best_sorted"], q_lab, img_scale, D)
        n_img = images.shape[0]
        if self.group is not None:
            allreduce_sum_([self.rhs, self.khat], self.group)
            if n_img not in self._n_total:
                self._n_total[n_img] = global_count(n_img, images.device, self.group)
            n_img = self._n_total[n_img]
        per_img = float(self.P2) if D is None else float(d_sum)
        lam = lam_rel * per_img * n_img
        x = self.plan.cg_solve(self.khat, lam, self.rhs, A, cg_iters, x=self.x, res_hist=res_hist)
        return res, x, lam

    def close(self):
        if self.sets:
            for _, s in self.sets:
                s.close()
        self.matcher.close()
        self.plan.close()
