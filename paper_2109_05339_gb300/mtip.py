"""One slice -> match -> merge -> CG iteration of M-TIP on one GPU (Fig. 3
without phasing), as a sequence of C-ABI calls.

1. Slicing (Sec. II-A) and matching (Sec. II-B), streamed in orientation
   chunks: each chunk of model images is sliced into one reusable buffer and
   matched against every image; the running top-k survives across chunks, so
   no more than one chunk of slices is ever resident.
2. Merging (Sec. II-C): type-1 right-hand side and Toeplitz kernel from the
   matched orientations, accumulated over image chunks (linearity, the
   paper's per-node type-1 sums followed by a reduction).
3. ``cg_iters`` conjugate-gradient steps on Eq. 2 from x0 = current model,
   lambda = lam_rel * sum of the weights D over all merged pixels.
"""
from __future__ import annotations

import torch

from .api import Matcher, Plan


class MTIP:
    def __init__(self, N, qmax, P2, n_img, n_orient, orient_chunk=None, img_chunk=None,
                 eps=1e-6, precision="bf16", topk=8, device=None):
        self.orient_chunk = min(n_orient, orient_chunk or n_orient)
        self.img_chunk = min(n_img, img_chunk or n_img)
        max_pts = max(self.orient_chunk, self.img_chunk) * P2
        self.plan = Plan(N, qmax, eps, max_points=max_pts, device=device)
        self.device = self.plan.device
        self.matcher = Matcher(n_img, self.orient_chunk, P2, precision, topk, device=self.device)
        dev = torch.device("cuda", self.device)
        self.slices = torch.empty((self.orient_chunk, P2), dtype=torch.float32, device=dev)
        self.rhs = torch.empty((N,) * 3, dtype=torch.float32, device=dev)
        self.khat = torch.empty((self.plan.PT,) * 3, dtype=torch.float32, device=dev)
        self.x = torch.empty((N,) * 3, dtype=torch.float32, device=dev)
        self.N, self.P2, self.n_img, self.n_orient = N, P2, n_img, n_orient

    def match(self, A, quats, q_lab, images, img_scale):
        m = self.matcher
        m.set_images(images, img_scale)
        M = quats.shape[0]
        for c0 in range(0, M, self.orient_chunk):
            c1 = min(M, c0 + self.orient_chunk)
            sl = self.slices[: c1 - c0]
            self.plan.slice_model(A, quats[c0:c1], q_lab, out=sl)
            m.add_slices(sl, orient_offset=c0)
        return m.results()

    def merge(self, images, quats, best, q_lab, img_scale, D=None):
        n = images.shape[0]
        for c0 in range(0, n, self.img_chunk):
            c1 = min(n, c0 + self.img_chunk)
            self.plan.merge_images(images[c0:c1], quats, q_lab, D=D, b_scale=img_scale, rhs=self.rhs,
                                   kernel_hat=self.khat, accumulate=c0 > 0, orient_idx=best[c0:c1])
        return self.rhs, self.khat

    def iteration(self, A, quats, q_lab, images, img_scale, cg_iters, lam_rel=1e-3, D=None,
                  d_sum=None, res_hist=None):
        """Returns (match results, merged model x, lambda); d_sum = sum of D over one image."""
        res = self.match(A, quats, q_lab, images, img_scale)
        self.merge(images, quats, res["best"], q_lab, img_scale, D)
        per_img = float(self.P2) if D is None else float(d_sum)
        lam = lam_rel * per_img * images.shape[0]
        x = self.plan.cg_solve(self.khat, lam, self.rhs, A, cg_iters, x=self.x, res_hist=res_hist)
        return res, x, lam

    def close(self):
        self.matcher.close()
        self.plan.close()
