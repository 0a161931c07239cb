#!/usr/bin/env python
"""Benchmark of one M-TIP slice -> match -> merge -> CG iteration on GB300.

A step is one pass of the whole path over one batch: slice the model at every
reference orientation (type-2 NUFFT), match every image against every slice
(cross term in BF16 on the tensor cores, FP32 re-rank of the top-8), merge the
images at their matched orientations (type-1 right-hand side and Toeplitz
kernel), and run the configured number of CG iterations.

Workload (default): 200-Gaussian density, 81^3 model, 128x128 Ewald detector,
10,000 orientations x 10,000 Poisson images at a mean of 1e3 photons/image,
10 CG iterations (synthetic, seeded; stands in for the paper's 3IYF data).

Prints one JSON line. `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CONFIG = "c2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16", "fp8", "fp32"], default="bf16")
    ap.add_argument("--config", default=CONFIG)
    ap.add_argument("--n-orient", type=int, default=None)
    ap.add_argument("--n-img", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fft-compare", action="store_true",
                    help="skip timing the Toeplitz apply against a cuFFT (torch.fft) version")
    ap.add_argument("--orient-chunk", type=int, default=None,
                    help="orientations sliced and matched per chunk (default: all at once)")
    ap.add_argument("--img-chunk", type=int, default=None,
                    help="images merged per type-1 call (default: all at once)")
    ap.add_argument("--compare-fp32", action="store_true",
                    help="also time the matching stage on the FP32 CUDA-core path")
    return ap.parse_args()


def workload_name(cfg, M, Ni):
    return (f"M-TIP iteration: {cfg.n_gauss}-Gaussian density, {cfg.N}^3 model, {cfg.P}x{cfg.P} "
            f"Ewald detector, {M} orientations x {Ni} images, {cfg.cg_iters} CG iterations")


# ------------------------------------------------------------------ clocks --
class Clocks:
    """nvidia-smi samples every 50 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# --------------------------------------------------------- roofline units --
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def traffic_for(kernel, units_per_launch):
    """DRAM bytes per launch from profiles/dram_traffic.json (ncu counters per
    unit of work), or None when no record exists or the kernel's source file
    changed since the counters were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
        return None
    return rec["dram_bytes_per_unit"] * units_per_launch


def roofline_for(kernel, launches, ms, ctx, peaks, src, clocks):
    """Algorithmic work per launch / average launch time, against its peak."""
    avg_s = ms / launches / 1e3
    if kernel.startswith("tc_match"):
        flops = 2.0 * ctx["n_img"] * ctx["n_orient_per_launch"] * ctx["P2"]
        peak = peaks["bf16_tflops_sustained"] * (2.0 if ctx["precision"] == "fp8" else 1.0)
        return {"kernel": kernel, "bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": f"{src} bf16 sustained" +
                (" x2 (fp8/bf16 nominal ratio)" if ctx["precision"] == "fp8" else "")}
    if kernel.startswith("simt_match"):
        flops = 2.0 * ctx["n_img"] * ctx["n_orient_per_launch"] * ctx["P2"]
        mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": "152 SMs x 128 FP32 lanes x 2 x median SM clock"}
    if kernel.startswith("interp") or kernel.startswith("spread"):
        # w^3 taps per point, one FP32 multiply-add each, against the SMs'
        # FP32 FMA rate (128 per clock per SM). The spreading accumulates taps
        # in registers; the tensor-core interpolation contracts the window on
        # the tensor cores and is bound by the per-point FP32 work around it.
        w = ctx["w"]
        pts = ctx["points_per_launch"][kernel.split("_")[0]]
        taps = pts * w ** 3
        mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * mhz * 1e6 / 1e9
        return {"kernel": kernel, "bound": "alu", "achieved": taps / avg_s / 1e9, "peak": peak,
                "unit": "Gtap/s",
                "peak_source": "152 SMs x 128 FP32 FMA/clock x median SM clock (one FMA per tap)"}
    # HBM-bound kernels: FFT passes etc.
    bytes_ = ctx.get("bytes_per_launch", {}).get(kernel)
    if bytes_ is None:
        return None
    return {"kernel": kernel, "bound": "hbm", "achieved": bytes_ / avg_s / 1e9,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "peak_source": f"{src} hbm"}


# --------------------------------------------------------------- our arm --
def run_ours(args, rank, world):
    import torch

    from paper_2109_05339_gb300 import build as _build
    _build.build()
    from paper_2109_05339_gb300 import _lib
    from paper_2109_05339_gb300.mtip import MTIP

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = synth.CONFIGS[args.config]
    M = args.n_orient or cfg.n_orient
    Ni = args.n_img or cfg.n_img
    pb = synth.make_problem(cfg, n_orient=M, n_img=Ni)
    P2 = pb.q_lab.shape[0]
    # inputs: model, orientations, detector (host, seeded), then the images:
    # noise-free slices at the image orientations -> global fluence -> Poisson
    A = torch.from_numpy(pb.A.astype(np.float32)).to(dev)
    quats = torch.from_numpy(pb.quats.astype(np.float32)).to(dev)
    qlab = torch.from_numpy(pb.q_lab.astype(np.float32)).to(dev)
    iq = torch.from_numpy(pb.img_quats.astype(np.float32)).to(dev)
    drv = MTIP(cfg.N, cfg.qmax, P2, Ni, M, orient_chunk=args.orient_chunk, img_chunk=args.img_chunk,
               eps=cfg.eps, precision=args.precision, device=dev,
               process_group=torch.distributed.group.WORLD if world > 1 else None)
    # noise-free slices at the image orientations, chunk by chunk
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg.seed * 1000 + rank)
    images = torch.empty((Ni, P2), dtype=torch.float32, device=dev)
    ch = drv.orient_chunk
    tot = 0.0
    for c0 in range(0, Ni, ch):
        drv.plan.slice_model(A, iq[c0:c0 + ch], qlab, out=images[c0:c0 + ch])
        tot += float(images[c0:c0 + ch].double().sum())
    s = cfg.photons / (tot / Ni)
    for c0 in range(0, Ni, ch):
        blk = images[c0:c0 + ch]
        blk.copy_(torch.poisson(blk * s, generator=gen))
    torch.cuda.synchronize()
    img_scale = 1.0 / s

    def step():
        return drv.iteration(A, quats, qlab, images, img_scale, cfg.cg_iters)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    # per-kernel table from a traced pass (event pair on every launch), kept
    # out of the timed region
    n_tr = max(1, min(args.steps, 5))
    _lib.profile_select(None)
    _lib.profile_enable(True)
    for _ in range(n_tr):
        step()
    torch.cuda.synchronize()
    prof_all = _lib.profile_read()
    _lib.profile_enable(False)
    dominant = max(prof_all.items(), key=lambda kv: kv[1][1])[0] if prof_all else None
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(dev.index)
    clocks.start()
    # timed region: events around the dominant kernel's launches only
    _lib.profile_select([dominant] if dominant else None)
    _lib.profile_enable(True)
    l0 = _lib.launch_count()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        res, x, lam = step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = _lib.launch_count() - l0
    prof = _lib.profile_read()
    _lib.profile_enable(False)
    _lib.profile_select(None)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    drv.plan.status()
    drv.matcher.status()

    # accuracy of this run's matching against its own exact re-rank is
    # implied; parity against the oracle lives in the tests.
    value = Ni * M * world / (ms / 1e3)
    # per-kernel table and the dominant kernel's roofline
    ctx = {"n_img": Ni, "n_orient_per_launch": drv.orient_chunk, "P2": P2, "precision": args.precision,
           "w": drv.plan.w, "points_per_launch": {
               "interp": drv.orient_chunk * P2,
               # class sums spread per cached orientation chunk; streaming
               # spreads the images of one image chunk
               "spread": (drv.orient_chunk if drv.cache_points else drv.img_chunk) * P2}}
    peaks, src = measured_peaks()
    kern = {k: {"launches": n / n_tr, "ms_per_step": t / n_tr} for k, (n, t) in prof_all.items()}
    roof = None
    if dominant and dominant in prof:
        n, t = prof[dominant]
        r = roofline_for(dominant, n, t, ctx, peaks, src, ck)
        if r:
            r["frac"] = r["achieved"] / r["peak"]
            units = (ctx["points_per_launch"].get(dominant.split("_")[0]) if dominant.startswith(("interp", "spread"))
                     else ctx["n_img"] * ctx["n_orient_per_launch"] if dominant.startswith(("tc_", "simt")) else None)
            r["traffic"] = traffic_for(dominant, units) if units else None
            roof = r
    stage = {}
    for k, v in kern.items():
        grp = ("slice" if k.startswith(("interp", "deconv_pad", "halo")) else
               "match" if k.startswith(("simt", "tc_", "rerank", "row_norms", "quantize", "state_reset",
                                        "results")) else
               "sort" if k.startswith(("key_", "scan_", "build_subs")) else
               "merge" if k.startswith(("spread", "crop_deconv", "crop_embed", "accumulate")) else
               "cg" if k.startswith(("pad_kernel", "crop_apply", "apply_kernel", "cg_", "finalize")) else
               "fft" if k.startswith("fft") else "other")
        stage[grp] = stage.get(grp, 0.0) + v["ms_per_step"]

    out = {
        "metric": "image x orientation matches/s (whole M-TIP iteration: slice + match + merge + CG)",
        "value": value, "unit": "matches/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16 cross term, f32 NUFFT/rerank, f64 CG dots",
                                       "fp8": "fp8 e4m3 cross term, f32 NUFFT/rerank, f64 CG dots",
                                       "fp32": "f32, f64 CG dots"}[args.precision],
        "data": "synthetic (seeded Gaussian density, Poisson images)",
        "config": {"workload": workload_name(cfg, M, Ni), "n_orient": M, "n_img": Ni, "N": cfg.N,
                   "detector": f"{cfg.P}x{cfg.P}", "cg_iters": cfg.cg_iters, "precision": args.precision,
                   "topk_rerank": 8, "nufft_eps": cfg.eps, "parallelism": f"dp{world} (image shards)",
                   "l2": (f"inputs larger than L2 (images {Ni * P2 * 4 / 1e6:.0f} MB, slices "
                          f"{drv.orient_chunk * P2 * 4 / 1e6:.0f} MB per chunk)"),
                   "orient_chunk": drv.orient_chunk,
                   "point_sets": "cached" if drv.cache_points else "streamed"},
        "nufft_mpts_per_s": {
            "slice_type2": (M * P2) / (stage.get("slice", 0) + 1e-12) / 1e3,
            "merge_type1_rhs_plus_kernel": (Ni * P2) / (stage.get("merge", 0) + 1e-12) / 1e3},
        "stage_ms": stage,
        "kernels": kern,
        "kernels_note": (f"per-kernel device time from a separate traced pass of {n_tr} steps; the timed "
                         "region records events around the dominant kernel only"),
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": ck,
    }
    if rank == 0 and not args.no_fft_compare:
        out["fft_vs_cufft"] = cufft_compare(drv, lam)
    if args.compare_fp32 and rank == 0:
        out["fp32_match"] = time_match_only(args, drv, A, quats, qlab, images, img_scale, "fp32")
        out["bf16_match"] = time_match_only(args, drv, A, quats, qlab, images, img_scale, args.precision)
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, drv, pb, images, img_scale, dev, M, Ni, world)
    return out, (pb, cfg)


def cufft_compare(drv, lam, reps=50):
    """The Toeplitz apply y = crop(IFFT(K^ FFT(pad x))) / PT^3 + lam x on the
    iteration's own kernel and model, through this library (hand-written
    real-input FFT passes) and through torch.fft (cuFFT; for comparison
    only): mean device ms per apply and the relative L2 difference."""
    import torch
    plan = drv.plan
    N, PT = plan.N, plan.PT
    khat, x = drv.khat, drv.x.clone()
    dev = khat.device
    idx = (torch.arange(N, device=dev) - (N - 1) // 2) % PT
    iz, iy, ix = idx[:, None, None], idx[None, :, None], idx[None, None, :]
    kh = khat[:, :, : PT // 2 + 1].contiguous()
    out = torch.empty_like(x)

    def ours():
        return plan.toeplitz_apply(khat, lam, x, out=out)

    def cufft():
        pad = torch.zeros((PT, PT, PT), dtype=torch.float32, device=dev)
        pad[iz, iy, ix] = x
        y = torch.fft.irfftn(torch.fft.rfftn(pad) * kh, s=(PT, PT, PT))
        return y[iz, iy, ix] + lam * x

    def timed(fn):
        for _ in range(3):
            fn()
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r.clone()

    t_ours, y_ours = timed(ours)
    t_lib, y_lib = timed(cufft)
    return {"op": f"Toeplitz apply: {N}^3 vector, {PT}^3 circulant embedding, real input",
            "ours_ms": t_ours, "cufft_ms": t_lib,
            "rel_l2_diff": float((y_ours - y_lib).norm() / y_lib.norm()),
            "note": "torch.fft (cuFFT) pad/rfftn/product/irfftn/crop, for comparison only; "
                    "L2-resident operands, CUDA events over the repeated applies"}


def time_match_only(args, drv, A, quats, qlab, images, img_scale, precision):
    """Matching stage alone (slices precomputed) for the FP32 vs BF16 comparison."""
    import torch
    from paper_2109_05339_gb300 import Matcher
    M = quats.shape[0]
    slices = drv.plan.slice_model(A, quats, qlab)
    m = Matcher(images.shape[0], M, images.shape[1], precision, 8, device=images.device)
    for _ in range(2):
        m.match(images, slices, img_scale)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        best, d1, d2 = m.match(images, slices, img_scale)
    e1.record()
    torch.cuda.synchronize()
    m.status()
    ms = e0.elapsed_time(e1) / reps
    out = {"ms": ms, "matches_per_s": images.shape[0] * M / (ms / 1e3), "best": best}
    m.close()
    del slices
    return {k: v for k, v in out.items() if k != "best"}


def run_e2e(args, drv, pb, images, img_scale, dev, M, Ni, world):
    """Same step through host buffers: H2D of the inputs and D2H of the results
    (best orientation per image, merged model) inside the timed region. The
    model and images of step i + 1 are copied on a second stream while step i
    computes (two device buffers); every step's copies stay inside the timed
    region. Integral images (photon counts) travel as 16-bit counts and the
    driver converts them to FP32 on the device inside the step."""
    import torch
    cfg = pb.cfg
    h_A = torch.from_numpy(pb.A.astype(np.float32)).pin_memory()
    h_q = torch.from_numpy(pb.quats.astype(np.float32)).pin_memory()
    h_l = torch.from_numpy(pb.q_lab.astype(np.float32)).pin_memory()
    # photon-count frames travel as 16-bit counts (the driver converts them on
    # the device inside the step); non-integral images would travel as FP32
    as_counts = bool(torch.equal(images, images.round())) and float(images.min()) >= 0.0 \
        and float(images.max()) <= 65535.0
    h_img = (images.to(torch.int32).to(torch.int16) if as_counts else images).cpu().pin_memory()
    d_q, d_l = torch.empty_like(h_q, device=dev), torch.empty_like(h_l, device=dev)
    d_A = [torch.empty_like(h_A, device=dev) for _ in range(2)]
    d_img = [torch.empty_like(h_img, device=dev) for _ in range(2)]
    o_best = torch.empty(Ni, dtype=torch.int32).pin_memory()
    o_x = torch.empty_like(h_A).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_A, h_q, h_l, h_img))
    d2h = o_best.numel() * 4 + o_x.numel() * 4
    comp = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def upload(b):
        with torch.cuda.stream(copy):
            copy.wait_event(freed[b])
            d_A[b].copy_(h_A, non_blocking=True)
            d_img[b].copy_(h_img, non_blocking=True)
            copied[b].record(copy)

    def run(n):
        for b in range(2):
            freed[b].record(comp)
        upload(0)
        for i in range(n):
            b = i % 2
            if i + 1 < n:
                upload(1 - b)
            d_q.copy_(h_q, non_blocking=True)
            d_l.copy_(h_l, non_blocking=True)
            comp.wait_event(copied[b])
            res, x, lam = drv.iteration(d_A[b], d_q, d_l, d_img[b], img_scale, cfg.cg_iters)
            o_best.copy_(res["best"], non_blocking=True)
            o_x.copy_(x, non_blocking=True)
            freed[b].record(comp)

    run(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    run(args.steps)
    e1.record(comp)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    return {"value": Ni * M * world / (ms / 1e3), "unit": "matches/s", "ms_per_step": ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "note": "inputs of step i+1 copied on a second stream while step i computes; images "
                    + ("as 16-bit photon counts, converted to FP32 on the device in the step" if as_counts
                       else "as FP32")}


# -------------------------------------------------------- oracle (CPU) ---
def oracle_sample(cfg, pb_full, m, n, reps=1):
    """Time the FP64 oracle's iteration on m orientations x n images of the
    same workload (full grid and detector), stage by stage."""
    from oracle import matching, merge, slicing
    from oracle.rotation import nufft_points
    rng = np.random.default_rng(123)
    quats = pb_full.quats[:m]
    iq = pb_full.img_quats[:n]
    t0 = time.perf_counter()
    sl = slicing.slice_model(pb_full.A, quats, pb_full.q_lab, cfg.qmax)
    t1 = time.perf_counter()
    # images: Poisson at the sample's own noise-free slices (input preparation, untimed)
    clean = slicing.slice_model(pb_full.A, iq, pb_full.q_lab, cfg.qmax)
    s = cfg.photons / float(np.mean(clean.sum(1)))
    X = rng.poisson(s * np.maximum(clean, 0)).astype(np.float64) / s
    t2 = time.perf_counter()
    res = matching.match(X, sl)
    t3 = time.perf_counter()
    N = cfg.N
    t = nufft_points(quats[res["best"]], pb_full.q_lab, N, cfg.qmax).reshape(-1, 3)
    D = np.ones(t.shape[0])
    lam = 1e-3 * t.shape[0]
    K = merge.toeplitz_kernel(t, D, N)
    Kh = merge.kernel_hat(K, N)
    bt = merge.rhs(X.ravel(), t, D, N, lam, pb_full.A)
    t4 = time.perf_counter()
    merge.cg(lambda v: merge.apply_toeplitz(v, Kh, N, lam), bt, pb_full.A, cfg.cg_iters)
    t5 = time.perf_counter()
    return {"slice": t1 - t0, "match": t3 - t2, "merge": t4 - t3, "cg": t5 - t4}


def extrapolate(st, m, n, M, Ni):
    """Full-workload oracle time from the sample: slicing scales with the
    orientations, matching with orientations x images, merging with the
    images, CG is fixed."""
    return st["slice"] * M / m + st["match"] * (M * Ni) / (m * n) + st["merge"] * Ni / n + st["cg"]


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    cfg = synth.CONFIGS[args.config]
    M = args.n_orient or cfg.n_orient
    Ni = args.n_img or cfg.n_img
    pb = synth.make_problem(cfg, n_orient=M, n_img=Ni)
    m = n = 2
    for _ in range(max(args.warmup, 0) and 1):
        oracle_sample(cfg, pb, m, n)
    tot = []
    for _ in range(args.steps):
        st = oracle_sample(cfg, pb, m, n)
        tot.append(extrapolate(st, m, n, M, Ni))
    t_full = float(np.median(tot))
    value = M * Ni / t_full
    sample = (f"{m} orientations x {n} images per step on the full {cfg.N}^3 grid and {cfg.P}x{cfg.P} "
              f"detector; per-stage times extrapolated linearly (slice x M, match x M*N, merge x N, CG fixed)")
    return {"impl": "reference", "metric": "image x orientation matches/s (whole M-TIP iteration: slice + "
            "match + merge + CG)", "value": value, "unit": "matches/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian density, Poisson images)",
            "config": {"workload": workload_name(cfg, M, Ni), "n_orient": M, "n_img": Ni},
            "cpu_baseline": {"value": value, "unit": "matches/s", "cores": cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "matches/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out, (pb, cfg) = run_ours(args, rank, world)
    if rank == 0 and not args.no_cpu_baseline:
        M, Ni = out["config"]["n_orient"], out["config"]["n_img"]
        m = n = 2
        st = oracle_sample(cfg, pb, m, n)
        t_full = extrapolate(st, m, n, M, Ni)
        out["cpu_baseline"] = {
            "value": M * Ni / t_full, "unit": "matches/s", "cores": cores(), "kind": "oracle",
            "sample": (f"FP64 oracle on {m} orientations x {n} images of this workload (full grid and "
                       f"detector, {cfg.cg_iters} CG), stage times {json.dumps({k: round(v, 2) for k, v in st.items()})} s "
                       f"extrapolated linearly to the full workload; numpy elementwise work single-threaded, "
                       f"BLAS on all cores")}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
