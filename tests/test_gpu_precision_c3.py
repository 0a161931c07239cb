"""The c3 precision study (c1 shapes: 17^3, 16 x 16, 500 orientations, 100
Poisson images, seed 3): argmin agreement of the FP32, BF16 and FP8 matching
paths (each with the FP32 re-rank of its top 8) with the FP64 oracle, per
oracle margin bin, on Poisson and on noise-free images; and the FP32 NUFFT
error against the FP64 direct sum on a 1e5-point subsample. The assertions
are the parity bars; the table is written as JSON to $SPF_REPORT_DIR when
that is set."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import matching, nudft, slicing
from oracle.rotation import nufft_points
from tests.gpu_util import f32, rel_l2, to_dev

pytestmark = pytest.mark.gpu
BINS = [0.0, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, np.inf]


def _match(precision, X, Y, scale):
    import torch
    from paper_2109_05339_gb300 import Matcher
    m = Matcher(X.shape[0], Y.shape[0], X.shape[1], precision, 8)
    best, _, _ = m.match(to_dev(X), to_dev(Y), float(scale))
    m.status()
    torch.cuda.synchronize()
    out = best.cpu().numpy()
    m.close()
    return out


def _table(best, ref):
    rows = []
    for lo, hi in zip(BINS[:-1], BINS[1:]):
        sel = (ref["margin"] >= lo) & (ref["margin"] < hi)
        row = {"margin_lo": lo, "margin_hi": None if np.isinf(hi) else hi, "images": int(sel.sum())}
        for p, b in best.items():
            row[p] = float(np.mean(b[sel] == ref["best"][sel])) if sel.any() else None
        rows.append(row)
    return rows


def test_c3_precision_study():
    pb = synth.make_problem("c3")
    Y = slicing.slice_model(pb.A, pb.quats, pb.q_lab, 1.0).astype(np.float32)
    clean = Y[pb.img_pick]
    counts, s = pb.image_counts(f32(clean))
    scale = np.float32(1.0 / s)
    report = {"config": "c3: 17^3 model, 16x16 detector, 500 orientations, 100 images, seed 3",
              "margin": "(d2 - d1) / (|x|^2 + |y_best|^2) of the FP64 oracle"}
    for kind, X, sc in (("poisson", counts, scale), ("noise_free", clean, np.float32(1.0))):
        Xd = f32(X) * np.float64(sc)
        ref = matching.match(Xd, f32(Y))
        best = {p: _match(p, X, Y, sc) for p in ("fp32", "bf16", "fp8")}
        report[kind] = _table(best, ref)
        ok = ref["margin"] > 1e-4
        for p in best:
            np.testing.assert_array_equal(best[p][ok], ref["best"][ok])
        if kind == "noise_free":
            np.testing.assert_array_equal(ref["best"], pb.img_pick)
            np.testing.assert_array_equal(best["fp32"], pb.img_pick)
            np.testing.assert_array_equal(best["bf16"], pb.img_pick)
            np.testing.assert_array_equal(best["fp8"], pb.img_pick)
            report["noise_free_exact"] = {p: float(np.mean(b == pb.img_pick)) for p, b in best.items()}
    # FP32 NUFFT (eps 1e-6) against the FP64 direct sum on 102,400 points
    from paper_2109_05339_gb300 import Plan
    q = pb.quats[:400].astype(np.float32)
    l32 = pb.q_lab.astype(np.float32)
    plan = Plan(pb.cfg.N, 1.0, 1e-6, max_points=400 * l32.shape[0])
    got = plan.slice_model(to_dev(pb.A.astype(np.float32)), to_dev(q), to_dev(l32)).cpu().numpy()
    plan.status()
    t = nufft_points(f32(q), f32(l32), pb.cfg.N, 1.0).reshape(-1, 3)
    ref = nudft.type2(f32(pb.A.astype(np.float32)), t).real
    err = rel_l2(got.ravel(), ref)
    report["nufft_fp32_vs_fp64_direct"] = {
        "points": int(t.shape[0]), "eps": 1e-6, "rel_l2": err,
        "max_abs_over_max_ref": float(np.max(np.abs(got.ravel() - ref)) / np.max(np.abs(ref)))}
    assert err < 1e-5, err
    plan.close()
    out = os.environ.get("SPF_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_c3.json"), "w") as fh:
            json.dump(report, fh, indent=1)
