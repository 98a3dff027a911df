#!/usr/bin/env python3
"""Benchmark of the w-stacking hot path: Mvis/s of the end-to-end image.

Default workload (one GPU): 16384^2 image, 32 w-planes, 1e8 visibilities from
300-station 8 h earth-rotation tracks over 64 channels (120-168 MHz), Gaussian
kernel W=7.  One step = bucket sort (wst_plan_set_vis) + gridding, per-plane 2D
FFT, phase screen, plane sum and grid correction (wst_image), inputs resident in
HBM.  Prints one JSON line (see the keys below).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|array|batched] [--chunk P]

--impl reference times the FP64 CPU oracle (the only CPU program of this method
here) on a bounded sample of the same workload.  Under torchrun every rank images
its own copy of the workload (replicas, weak scaling); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mvis/s end-to-end w-stacking image (16384², 32 planes) + max err vs FP64 DFT"
HBM_FALLBACK_GBS = 6800.0

WORKLOADS = {
    "large": "16384^2 image, 32 w-planes, 1e8 visibilities (300 stations, 8 h tracks at dec +45, "
             "64 channels 120-168 MHz, 35 dumps), FoV 0.5 rad, Gaussian W=7 sigma=0.875",
    "array": "4096^2 image, 32 w-planes, 4.08e6 visibilities (60 stations, 144 dumps, 16 channels), "
             "FoV 0.2 rad, Gaussian W=7",
    "batched": "64 channel images of 2048^2, 16 w-planes each, 1e5-2e6 visibilities per image (log-uniform), "
               "FoV 0.09 rad, Gaussian W=7",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--chunk", type=int, default=0, help="planes per chunk (0 = all planes resident)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison of the transform stage")
    ap.add_argument("--shard", choices=["replicas", "planes"], default="replicas",
                    help="replicas: every rank images its own copy of the workload (weak scaling); planes: the "
                         "ranks split one job's w-planes and sum the partial images with one all-reduce "
                         "(strong scaling)")
    ap.add_argument("--dft-pixels", type=int, default=64)
    ap.add_argument("--n-w", type=int, default=0, help="override the number of w-planes (profiling cases)")
    ap.add_argument("--vis-frac", type=float, default=1.0, help="keep this fraction of the visibilities")
    ap.add_argument("--snap-w", action="store_true",
                    help="place every w on its plane centre, so the error against the direct transform is "
                         "the (u,v) kernel's alone (kernel comparisons)")
    ap.add_argument("--table-per-cell", type=int, default=1024,
                    help="samples per cell of the tabulated kernels (kb8, learned); 1024 is the trained "
                         "kernel's resolution, 128 keeps the gridder's tap table in L1 (3%% faster)")
    ap.add_argument("--image-n", type=int, default=0,
                    help="image the central N pixels of the workload's field (FoV N/n, the same pixels) on "
                         "its n-cell grid: oversampling n/N (e.g. 3276 of 4096: 1.25); 0 = the whole field")
    ap.add_argument("--oversample", type=int, default=0, choices=[0, 1, 2],
                    help="2: grid of 2N cells, the central N x N kept (images up to 8192^2)")
    ap.add_argument("--wfold", action="store_true",
                    help="mirror w < 0 visibilities (WST_FLAG_WFOLD): half the w range; the real part is the image")
    ap.add_argument("--kernel", choices=["gauss", "learned", "gauss8", "es8", "kb8", "pswf8"], default="gauss",
                    help="gauss: W=7 Gaussian (the paper's); W=8 kernels: gauss8 Gaussian (sigma 0.925), es8 "
                         "exponential of semicircle (beta 2.3 W), kb8 Kaiser-Bessel table (beta of Beatty et "
                         "al. for the grid's oversampling), pswf8 prolate spheroidal table (c = pi W (1 - "
                         "1/(2 alpha))), learned the trained table "
                         "(paper_2301_06061_gb300/data/learned_kernel_w8.npz)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------------------------------------
# workloads (seeded, synthetic; see paper_2301_06061_gb300/synth.py)
# ------------------------------------------------------------------------------------------

def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mvis(world: int, n_vis: int, ms: float) -> float:
    """Whole-job throughput in Mvis/s: every rank images its own n_vis visibilities in ms."""
    return world * n_vis / (ms * 1e-3) / 1e6


def make_workload(name: str, rank: int, n_w: int = 0, vis_frac: float = 1.0):
    from paper_2301_06061_gb300 import synth

    if name == "large":
        work = synth.large(n_vis=int(100_000_000 * vis_frac), seed_extra=rank)
    elif name == "array":
        work = synth.array(seed_extra=rank)
    else:
        work = synth.batched(seed_extra=rank)
    if n_w > 0:
        work.n_w = n_w
    if work.sky is None:  # 200 point sources, dN/dS ~ S^-2 on [0.01, 1] Jy, inside 80% of the field
        work.sky = synth.power_law_sky(200, 0.4 * work.fov, 0.01, 1.0, synth.rng_for(3, 900 + rank))
    return work


def random_values(work, rank: int):
    """Seeded complex Gaussian values: the oracle's work does not depend on the values."""
    from paper_2301_06061_gb300 import synth

    return synth.random_visibilities(work.n_vis, synth.rng_for(3, 7 + rank))


# ------------------------------------------------------------------------------------------
# accuracy against the direct transform, with the stated per-pixel bound
# ------------------------------------------------------------------------------------------

def kernel_function(kernel: str, support: int, sigma: float, table):
    """(G, quadrature panels) of a kernel: a tabulated one (learned, kb8, pswf8) interpolated
    linearly as the library does, es8's exponential of semicircle (sigma holds beta), or
    the Gaussian."""
    half = 0.5 * support
    if table is not None:
        nodes = np.linspace(-half, half, table.size)
        return lambda t: np.interp(t, nodes, table.astype(np.float64)), table.size - 1
    if kernel == "es8":
        return (lambda t: np.where(np.abs(t) <= half,
                                   np.exp(sigma * (np.sqrt(np.clip(1.0 - (t / half) ** 2, 0.0, None)) - 1.0)), 0.0),
                support * 64)
    return lambda t: np.exp(-t * t / (2.0 * sigma * sigma)), support * 64


def kernel_error(kernel: str, support: int, sigma: float, table, n: int, idx: np.ndarray,
                 n_offsets: int = 512, oversample: float = 1) -> np.ndarray:
    """eps(a) = sup over sub-cell offsets g of |sum_taps G(t) e^{2 pi i nu t} / Ghat(nu) - 1|,
    t = tap - W/2 + g, nu = (a - n/2)/(oversample n): the relative error of one
    visibility's gridded, transformed and corrected contribution at pixel index a along
    one axis (an oversampled grid keeps the pixels in |nu| <= 1/(2 oversample))."""
    G, panels = kernel_function(kernel, support, sigma, table)
    half = 0.5 * support
    nu = (idx.astype(np.float64) - n // 2) / (n * oversample)
    # Ghat(nu) = integral of G(t) cos(2 pi nu t) over the support: 4-point Gauss-Legendre per panel
    gx, gw = np.polynomial.legendre.leggauss(4)
    edges = np.linspace(-half, half, panels + 1)
    h = edges[1] - edges[0]
    t = (edges[:-1, None] + 0.5 * h * (gx[None, :] + 1.0)).ravel()
    wq = np.tile(0.5 * h * gw, panels)
    gq = G(t) * wq
    ghat = np.array([np.sum(gq * np.cos(2.0 * np.pi * x * t)) for x in nu])
    g = (np.arange(n_offsets) + 0.5) / n_offsets
    taps = np.arange(support)[None, :] - half + g[:, None]  # (offsets, W)
    gt = G(taps)
    eps = np.empty(nu.size)
    for i, x in enumerate(nu):
        s = np.sum(gt * np.exp(2j * np.pi * x * taps), axis=1) / ghat[i]
        eps[i] = np.abs(s - 1.0).max()
    return eps


def accuracy_block(torch, wst, work, plan_stats, d_u, d_v, d_w, d_vis, img, dev, n_pix: int, kernel: str,
                   support: int, sigma: float, table, wfold: bool = False, oversample: float = 1, plan=None,
                   n_img: int = 0, fov_img: float = 0.0):
    """The image against the direct transform (GPU, float-float phases) at the brightest
    sources' pixels and at seeded random pixels, with the per-pixel bound
    B = sum|V| (min(2, 2 pi dmax |n - 1|) + e_a + e_b + e_a e_b) + 1e-5 peak, dmax the
    largest distance of a w from its plane centre and e the kernel error above.  With
    w-folding the real parts are compared (the folded image's real part is the dirty
    image) and the plane offsets are those of |w|.  n_img, fov_img: the image's side and
    field when they are not the workload's (an image cropped from the workload's grid)."""
    n, fov = (n_img, fov_img) if n_img else (work.n, work.fov)
    sky = work.sky
    order = np.argsort(-sky.flux)[: n_pix // 2]
    sa = np.clip(np.rint(n // 2 + sky.l[order] * n / fov), 0, n - 1).astype(np.int64)
    sb = np.clip(np.rint(n // 2 + sky.m[order] * n / fov), 0, n - 1).astype(np.int64)
    rng = np.random.default_rng(20230106)
    q = n_pix - sa.size
    ra = np.concatenate([rng.integers(3 * n // 8, 5 * n // 8, q // 2), rng.integers(0, n, q - q // 2)])
    rb = np.concatenate([rng.integers(3 * n // 8, 5 * n // 8, q // 2), rng.integers(0, n, q - q // 2)])
    pa, pb = np.concatenate([sa, ra]), np.concatenate([sb, rb])
    d_pa = torch.from_numpy(pa.astype(np.int32)).to(dev)
    d_pb = torch.from_numpy(pb.astype(np.int32)).to(dev)
    dft = torch.empty(pa.size, dtype=torch.complex64, device=dev)
    # the direct transform of the visibilities the image holds: those the sort dropped
    # (footprint off the grid) or found non-finite get weight 0
    kept = None
    if plan is not None:
        k = torch.empty(d_u.numel(), dtype=torch.int32, device=dev)
        i0, j0 = torch.empty_like(k), torch.empty_like(k)
        wst.wst_vis_cells(plan.handle, k, i0, j0)
        kept = (k >= 0).float()
        del k, i0, j0
    wst.wst_dft(d_u, d_v, d_w, d_vis, n, fov, d_pa, d_pb, dft, weight=kept)
    got = img[0][d_pb.long(), d_pa.long()]
    if wfold:
        err = (got.real - dft.real).abs().double().cpu().numpy()
        dft_abs = dft.real.abs().double().cpu().numpy()
    else:
        err = (got - dft).abs().double().cpu().numpy()
        dft_abs = dft.abs().double().cpu().numpy()
    peak = dft_abs.max()
    sum_abs = float((d_vis.abs().double() * (1.0 if kept is None else kept.double())).sum().item())
    # largest |w - w_k| over the data, w_k the centre of the plane the visibility lands on
    lo, hi = float(plan_stats["w_min"]), float(plan_stats["w_max"])
    w64 = d_w.double().abs() if wfold else d_w.double()
    k = torch.clamp(torch.floor((w64 - lo) * (work.n_w / (hi - lo))), 0, work.n_w - 1)
    dmax = float((w64 - (lo + (k + 0.5) * (hi - lo) / work.n_w)).abs().max().item())
    la = (pa - n // 2) * fov / n
    mb = (pb - n // 2) * fov / n
    r2 = la * la + mb * mb
    nm1 = np.abs(r2 / (1.0 + np.sqrt(np.maximum(0.0, 1.0 - r2))))
    ea = kernel_error(kernel, support, sigma, table, n, pa, oversample=oversample)
    eb = kernel_error(kernel, support, sigma, table, n, pb, oversample=oversample)
    rel = np.minimum(2.0, 2.0 * np.pi * dmax * nm1) + ea + eb + ea * eb
    bound = sum_abs * rel + 1e-5 * peak
    central = (np.abs(pa - n // 2) < n // 8) & (np.abs(pb - n // 2) < n // 8)
    inner = (np.abs(pa - n // 2) < 3 * n // 8) & (np.abs(pb - n // 2) < 3 * n // 8)  # central 3/4
    return {"reference": "wst_dft (GPU direct transform of Eq. 2 with float-float phases) of the gridded "
                         "visibilities (dropped ones excluded)",
            "excluded_visibilities": None if kept is None else int(kept.numel() - kept.sum().item()),
            "sky": f"{sky.flux.size} point sources, visibilities by Eq. 1 (wst_predict_points)",
            "pixels": int(pa.size), "source_pixels": int(sa.size),
            "max_err_rel_peak": float(err.max() / peak),
            "central_max_err_rel_peak": float(err[central].max() / peak) if central.any() else None,
            "inner3q_max_err_rel_peak": float(err[inner].max() / peak) if inner.any() else None,
            "inner3q_rms_err_rel_peak": float(np.sqrt(np.mean(err[inner] ** 2)) / peak) if inner.any() else None,
            "max_err_over_bound": float((err / bound).max()),
            "bound_rel_peak": {"min": float(bound.min() / peak), "median": float(np.median(bound) / peak),
                               "max": float(bound.max() / peak)},
            "w_offset_max": dmax,
            "kernel_error_max": float(max(ea.max(), eb.max())),
            "bound": "per pixel: sum|V| (min(2, 2 pi dmax |n-1|) + e_a + e_b + e_a e_b) + 1e-5 peak; e = sup over "
                     "sub-cell offsets of the corrected one-visibility error of the kernel at that pixel"}


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# roofline bookkeeping
# ------------------------------------------------------------------------------------------

def stage_bytes(stage: str, n: int, planes: int, chunks: int, batch: int, n_kept: int, n_vis: int,
                oversample: int = 1) -> float:
    """Algorithmic DRAM bytes of one launch of a stage (averaged over the chunks); the
    planes are (oversample n)^2, the images n^2."""
    S_img = 8.0 * n * n
    S = S_img * oversample * oversample
    per_chunk_planes = planes / chunks
    if stage == "sort":  # read u, v, w, V (20 B) and write the 32-byte record
        return 52.0 * n_vis
    if stage == "grid":  # write every plane cell once, read the 32-byte records once
        return per_chunk_planes * S + 32.0 * n_kept / chunks
    if stage in ("rows", "cols_a"):  # read + write each plane
        return 2.0 * per_chunk_planes * S
    if stage == "cols_b":  # read each plane, write the images once
        return per_chunk_planes * S + batch * S_img / chunks
    raise ValueError(stage)


def step_roofline(stage_ms: dict, n: int, planes: int, chunks: int, batch: int, n_kept: int, n_vis: int,
                  oversample: int, ms_step: float, peak: float) -> dict:
    """The whole step against HBM: the algorithmic bytes of every stage that ran (per
    step), and the all-resident floor of 4 S per plane (grid write, two column passes
    that read and write, counted as S + 2S + S) plus one image write."""
    launches = {"sort": 1, "grid": chunks, "rows": chunks, "cols_a": chunks, "cols_b": chunks}
    total = sum(stage_bytes(k, n, planes, chunks, batch, n_kept, n_vis, oversample) * launches[k]
                for k, ms in stage_ms.items() if ms > 0)
    floor = 4.0 * planes * 8.0 * (n * oversample) ** 2 + batch * 8.0 * n * n
    sec = ms_step * 1e-3
    return {"bytes": total, "ms": round(ms_step, 3), "achieved": round(total / sec / 1e9, 1),
            "frac": round(total / sec / 1e9 / peak, 4), "all_resident_floor_bytes": floor,
            "frac_of_all_resident_floor": round(floor / sec / 1e9 / peak, 4)}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2301_06061_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2301_06061_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_ratios():
    """Per plane kernel, DRAM bytes measured by ncu on the small 16384^2 case over that
    kernel's design bytes on the same case (profiles/traffic_16384_small.md), if the file
    was taken with these CUDA sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic_16384_small.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m_hash or m_hash.group(1) != kernel_source_hash():
        return None
    out = {}
    for key in ("grid_read", "grid_write", "cols_a_read", "cols_a_write", "cols_b_read", "cols_b_write"):
        m = re.search(rf"{key}_ratio:\s*([0-9.eE+-]+)", text)
        if not m:
            return None
        out[key] = float(m.group(1))
    return out


def launch_traffic(stage: str, n: int, planes_per_launch: float, rows_gridded_per_launch: float, n_kept_per_launch: float,
                   images: int, oversample: int = 1, ratios: dict | None = None):
    """DRAM bytes of one launch of a plane kernel: its design bytes on this workload (the
    occupied rows it writes or reads, the records, the planes, the image) times the ratio
    of measured to design bytes of the small-case capture; None without a matching
    capture.  The design bytes scale with the units each kernel moves, so the ratios do."""
    r = traffic_ratios() if ratios is None else ratios
    if r is None or stage not in ("grid", "cols_a", "cols_b"):
        return None
    row = 8.0 * n * oversample
    S = row * n * oversample
    if stage == "grid":
        return r["grid_read"] * 32.0 * n_kept_per_launch + r["grid_write"] * row * rows_gridded_per_launch
    if stage == "cols_a":
        return r["cols_a_read"] * row * rows_gridded_per_launch + r["cols_a_write"] * S * planes_per_launch
    return r["cols_b_read"] * S * planes_per_launch + r["cols_b_write"] * 8.0 * n * n * images


# ------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline leg and --impl reference)
# ------------------------------------------------------------------------------------------

ORACLE_SAMPLE_MAX_VIS = 4_000_000


def oracle_sample(work, vis, plane: int):
    """One w-plane of the workload with (a seeded subset of at most 4M of) its
    visibilities, as an n_w = 1 oracle problem on the full image."""
    import oracle

    lo, hi = oracle.resolve_w_range(work.w, work.w_min, work.w_max) if work.batch_offsets is None else (0, 0)
    full = oracle.OracleConfig(work.n, work.fov, work.n_w, lo, hi, work.support, "gauss", 0.875)
    k, _, _, st = oracle.locate(full, work.u, work.v, work.w, vis)
    sel = np.nonzero((st == 0) & (k == plane))[0]
    if sel.size > ORACLE_SAMPLE_MAX_VIS:
        sel = np.sort(np.random.default_rng(2301).choice(sel, ORACLE_SAMPLE_MAX_VIS, replace=False))
    dw = (hi - lo) / work.n_w
    cfg = oracle.OracleConfig(work.n, work.fov, 1, lo + plane * dw, lo + (plane + 1) * dw, work.support,
                              "gauss", 0.875)
    return cfg, work.u[sel], work.v[sel], work.w[sel], vis[sel]


def oracle_job_seconds(t_grid: float, t_image: float, n_sample: int, n_vis: int, n_w: int) -> float:
    """The whole job's oracle time from one sample plane: gridding scales with the
    visibilities, the transform, screen and plane sum with the planes.  The sample's
    image time t_image = t_grid + t_rest (one plane's FFT, screen, sum and the final
    correction), so job = (n_vis / n_sample) t_grid + n_w t_rest (which bills the
    correction, an elementwise pass, once per plane: an upper bound)."""
    t_rest = max(t_image - t_grid, 0.0)
    return (n_vis / max(n_sample, 1)) * t_grid + n_w * t_rest


def time_oracle_sample(work, vis, repeats: int = 1):
    """Seconds per full job, extrapolated from one plane of the single-image workloads by
    oracle_job_seconds; also the seconds this sample took, a description, the thread
    count, and the sample with the oracle's image of it."""
    import oracle

    plane = work.n_w // 2
    cfg, u, v, w, vv = oracle_sample(work, vis, plane)
    tg, ti = [], []
    ref = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.grid(cfg, u, v, w, vv)
        t1 = time.perf_counter()
        ref = oracle.image(cfg, u, v, w, vv)
        t2 = time.perf_counter()
        tg.append(t1 - t0)
        ti.append(t2 - t1)
    t_grid, t_image = statistics.median(tg), statistics.median(ti)
    job_s = oracle_job_seconds(t_grid, t_image, u.size, work.n_vis, work.n_w)
    sample = (f"w-plane {plane} of {work.n_w}: {u.size} of its visibilities (of {work.n_vis}), {work.n}^2 FP64 "
              f"grid, FFT, screen, correction; gridding alone {t_grid:.2f} s, the plane's image {t_image:.2f} s")
    extrap = {"formula": "job_s = (n_vis / n_sample) * t_grid + n_w * (t_image - t_grid)",
              "n_vis": work.n_vis, "n_sample": int(u.size), "n_w": work.n_w, "t_grid_s": round(t_grid, 4),
              "t_image_s": round(t_image, 4), "job_s": round(job_s, 3)}
    measured_s = (sum(tg) + sum(ti)) / repeats  # seconds this sample took per repeat
    return job_s, sample, oracle.num_threads(), (cfg, u, v, w, vv, ref), extrap, measured_s


def oracle_parity(torch, wst, dev, sample):
    """The CUDA path on the oracle's sample (same plane slab, n_w = 1) against the oracle's
    FP64 image: max error over the central half (|nu| <= 1/4) and over the whole image,
    relative to the peak."""
    cfg, u, v, w, vv, ref = sample
    c = wst.Config(n=cfg.n, fov=cfg.fov, n_w=1, w_min=cfg.w_min, w_max=cfg.w_max, support=cfg.support,
                   kparam=cfg.kparam, flags=wst.WST_FLAG_KAHAN)
    plan = wst.Plan(c, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    plan.set_vis(t(u), t(v), t(w), t(vv))
    img = plan.image()[0].cpu().numpy().astype(np.complex128)
    plan.close()
    n = cfg.n
    err = np.abs(img - ref)
    q = slice(n // 4, 3 * n // 4)
    peak = np.abs(ref).max()
    return {"sample": f"w-plane slab of the workload, {u.size} visibilities, {n}^2, full image",
            "central_half_max_err_rel_peak": float(err[q, q].max() / np.abs(ref[q, q]).max()),
            "max_err_rel_peak": float(err.max() / peak)}


# ------------------------------------------------------------------------------------------
# cuFFT as a yardstick for the transform stage (comparison only, never on the product path)
# ------------------------------------------------------------------------------------------

def centred_fft_cufft(torch, planes):
    """The centred, unnormalised, positive-exponent 2D transform of Eq. 2 by cuFFT
    (torch.fft): F = (-1)^(a+b) IFFT2((-1)^(p+q) g) without the 1/N^2 (N divisible by 4)."""
    n = planes.shape[-1]
    idx = torch.arange(n, device=planes.device)
    sign = (1 - 2 * ((idx[:, None] + idx[None, :]) & 1)).to(planes.real.dtype)
    return torch.fft.ifft2(planes * sign, norm="forward") * sign


def cufft_compare(torch, wst, plan, work, dev, stage_ms_per_plane: dict, peak: float, n_planes: int = 2):
    """Planes of the benchmark (wst_grid) transformed by cuFFT and by this library's
    transform stage, timed and compared.  This library's plain transform comes from
    wst_fft_correct on a one-plane plan whose plane centre is w = 0 (screen exactly 1)."""
    n = work.n
    p0 = work.n_w // 2
    g = torch.empty((n_planes, n, n), dtype=torch.complex64, device=dev)
    wst.wst_grid(plan.handle, p0, p0 + n_planes, g)
    stream = torch.cuda.current_stream(dev)
    out = centred_fft_cufft(torch, g)  # warm-up (plans cuFFT)
    del out
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        out = torch.fft.ifft2(g, norm="forward")  # the transform alone (no centring signs)
        del out
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_plane = e0.elapsed_time(e1) / reps / n_planes
    S = 8.0 * n * n
    ref = centred_fft_cufft(torch, g[:1])[0]
    zero = wst.Plan(wst.Config(n=n, fov=work.fov, n_w=1, w_min=-1.0, w_max=1.0, flags=wst.WST_FLAG_KAHAN),
                    device=dev)
    e = torch.empty(0, dtype=torch.float32, device=dev)
    zero.set_vis(e, e, e, torch.empty(0, dtype=torch.complex64, device=dev))
    ours = torch.zeros((1, n, n), dtype=torch.complex64, device=dev)
    wst.wst_fft_correct(zero.handle, 0, 1, g[:1].contiguous(), ours)
    diff = float((ours[0] - ref).abs().max() / ref.abs().max())
    zero.close()
    del g, ref, ours
    ours_ms = sum(stage_ms_per_plane.values())
    return {"what": "cuFFT (torch.fft.ifft2, c2c FP32, out of place) on planes of this workload, against this "
                    "library's transform stage (row FFT inside the gridding kernel, column stages A and B)",
            "n": n, "planes_timed": n_planes, "cufft_ms_per_plane": round(ms_plane, 4),
            "cufft_gbs_on_4S": round(4 * S / (ms_plane * 1e-3) / 1e9, 1),
            "cufft_frac_of_hbm_on_4S": round(4 * S / (ms_plane * 1e-3) / 1e9 / peak, 4),
            "ours_ms_per_plane": {k: round(v, 4) for k, v in stage_ms_per_plane.items()},
            "ours_total_ms_per_plane": round(ours_ms, 4),
            "ours_note": "the row pass is fused with gridding and column stage B with the phase screen and the "
                         "plane sum, so these include work cuFFT does not do",
            "max_diff_rel_peak": diff,
            "diff_of": "centred transform of one plane: wst_fft_correct on a one-plane plan with w_k = 0 vs cuFFT"}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def run_ours(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_2301_06061_gb300 import build, wst

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build.build()
    work = make_workload(args.workload, rank, args.n_w, args.vis_frac)
    if args.snap_w:
        lo, hi = float(work.w.min()), float(work.w.max())
        k = np.clip(np.floor((work.w.astype(np.float64) - lo) * (work.n_w / (hi - lo))), 0, work.n_w - 1)
        work.w = (lo + (k + 0.5) * (hi - lo) / work.n_w).astype(np.float32)
        work.w_min, work.w_max = lo, hi
        work.rows_m = work.chan_scale = None  # snapped w no longer follow the rows
    n_vis = work.n_vis
    batch = 1 if work.batch_offsets is None else len(work.batch_offsets) - 1
    dev = torch.device("cuda", local_rank)
    table = None
    if args.kernel == "gauss":
        kcfg = dict(support=work.support, kparam=wst.DEFAULT_SIGMA[work.support])
    elif args.kernel == "gauss8":
        kcfg = dict(support=8, kparam=wst.DEFAULT_SIGMA[8])
    elif args.kernel == "es8":
        kcfg = dict(support=8, kernel=wst.WST_KERNEL_ES, kparam=2.3 * 8)
    else:
        if args.kernel in ("kb8", "pswf8"):
            from paper_2301_06061_gb300 import kernels

            alpha = work.n / args.image_n if args.image_n else float(max(1, args.oversample))
            if args.kernel == "kb8":
                tab_np = kernels.kaiser_bessel_table(8, kernels.kaiser_bessel_beta(8, alpha), args.table_per_cell)
            else:
                tab_np = kernels.pswf_table(8, kernels.pswf_c(8, alpha), args.table_per_cell)
        else:
            from paper_2301_06061_gb300 import learned

            tab_np = learned.table_at(os.path.join(ROOT, "paper_2301_06061_gb300", "data", "learned_kernel_w8.npz"),
                                      args.table_per_cell)
        table = torch.from_numpy(tab_np).to(dev)
        kcfg = dict(support=8, kernel=wst.WST_KERNEL_TABLE, kparam=0.0, ktable_len=int(tab_np.size))
    # the image: the whole field on n pixels (or 2n grid cells with --oversample 2), or
    # with --image-n the central N pixels (field FoV N/n) on the workload's n-cell grid
    if args.image_n:
        if args.oversample == 2 or args.image_n % 2 or not 64 <= args.image_n <= work.n:
            raise SystemExit("--image-n: an even N, 64 <= N <= the workload's n, without --oversample 2")
        img_n, img_fov, grid_n, osf = args.image_n, work.fov * args.image_n / work.n, work.n, work.n / args.image_n
    else:
        img_n, img_fov, grid_n, osf = work.n, work.fov, 0, float(max(1, args.oversample))
    cfg = wst.Config(n=img_n, fov=img_fov, n_w=work.n_w, w_min=work.w_min, w_max=work.w_max,
                     flags=wst.WST_FLAG_KAHAN | wst.WST_FLAG_TIMING | (wst.WST_FLAG_WFOLD if args.wfold else 0),
                     planes_per_chunk=args.chunk, batch=batch, oversample=args.oversample, grid_n=grid_n,
                     **kcfg)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_u, h_v, h_w = pin(work.u), pin(work.v), pin(work.w)
    d_u, d_v, d_w = (t.to(dev) for t in (h_u, h_v, h_w))
    # the visibilities of the workload's point-source sky (Eq. 1), predicted on the GPU
    d_vis = torch.empty(n_vis, dtype=torch.complex64, device=dev)
    sky_t = [torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
             for a in (work.sky.l, work.sky.m, work.sky.flux)]
    wst.wst_predict_points(d_u, d_v, d_w, *sky_t, d_vis)
    h_vis = d_vis.cpu().pin_memory()
    vis_np = h_vis.numpy()
    offsets = None if work.batch_offsets is None else [int(x) for x in work.batch_offsets]
    plan = wst.Plan(cfg, device=dev)
    if table is not None:
        plan.set_kernel_table(table)
    img = torch.empty((batch, img_n, img_n), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.set_vis(d_u, d_v, d_w, d_vis, None, offsets)
        plan.image(out=img)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    plan.stats()  # drop warm-up timings
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    st = plan.stats()
    ms_step = max_over_ranks(ms_total / args.steps, dist, dev)
    value = job_mvis(world, n_vis, ms_step)

    # stage times inside the timed region (CUDA events on the plan's stream)
    stages = {"sort": st["ms_sort"], "grid": st["ms_grid"], "rows": st["ms_rows"], "cols_a": st["ms_cols_a"],
              "cols_b": st["ms_cols_b"]}
    launches_per_stage = {"sort": 1, "grid": st["n_chunks"], "rows": st["n_chunks"], "cols_a": st["n_chunks"],
                          "cols_b": st["n_chunks"]}
    dom = max(stages, key=stages.get)
    per_launch_ms = stages[dom] / (args.steps * launches_per_stage[dom])
    planes = batch * work.n_w
    peak, peak_src = load_peaks()
    kernel_names = {"sort": "k_keys+k_scan+k_scatter+k_row_bounds", "grid": "k_grid_rows (gridding + row FFT)",
                    "rows": "k_rows", "cols_a": "k_cols_a16 (column stage A)",
                    "cols_b": "k_cols_b_tma (column stage B + phase screen + compensated plane sum)"}
    # algorithmic bytes of a launch: what this design must move -- the occupied rows the
    # gridder writes and column stage A reads (rows no visibility reaches are known zero
    # and never touched), the records, the planes and the image.  The nominal bytes
    # (every row of every plane written and read, as a gridder without the occupancy
    # would) are reported beside them.
    ones = {k: 1.0 for k in ("grid_read", "grid_write", "cols_a_read", "cols_a_write", "cols_b_read", "cols_b_write")}

    def needed_bytes(stage):
        b = launch_traffic(stage, img_n, planes / st["n_chunks"], st["n_rows_gridded"] / st["n_chunks"],
                           st["n_kept"] / st["n_chunks"], batch, osf, ratios=ones)
        return stage_bytes(stage, img_n, planes, st["n_chunks"], batch, st["n_kept"], n_vis, osf) if b is None else b

    def frac(nbytes, ms):
        return round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)

    bytes_launch = needed_bytes(dom)
    nominal = stage_bytes(dom, img_n, planes, st["n_chunks"], batch, st["n_kept"], n_vis, osf)
    achieved = bytes_launch / (per_launch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kernel_names[dom], "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": launch_traffic(dom, img_n, planes / st["n_chunks"], st["n_rows_gridded"] / st["n_chunks"],
                                          st["n_kept"] / st["n_chunks"], batch, osf),
                "traffic_source": "small-case ncu ratios (profiles/traffic_16384_small.md) times this launch's "
                                  "design bytes (n_rows_gridded occupied rows, records, planes, image)",
                "bytes_per_launch": bytes_launch, "bytes": "occupied rows, records, planes, image (this design)",
                "ms_per_launch": round(per_launch_ms, 4),
                "nominal_bytes_per_launch": nominal, "nominal_frac": frac(nominal, per_launch_ms),
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "stage_ms_per_step": {k: round(v / args.steps, 4) for k, v in stages.items()},
                "stage_frac_of_hbm": {k: frac(needed_bytes(k) * launches_per_stage[k], v / args.steps)
                                      for k, v in stages.items() if v > 0},
                "stage_frac_of_hbm_nominal": {
                    k: frac(stage_bytes(k, img_n, planes, st["n_chunks"], batch, st["n_kept"], n_vis, osf) *
                            launches_per_stage[k], v / args.steps) for k, v in stages.items() if v > 0}}
    roofline["step"] = step_roofline({k: v / args.steps for k, v in stages.items()}, img_n, planes,
                                     st["n_chunks"], batch, st["n_kept"], n_vis, osf, ms_step, peak)
    # the step on this design's bytes (the nominal sum above counts every row of every plane)
    step_needed = sum(needed_bytes(k) * launches_per_stage[k] for k, v in stages.items() if v > 0)
    roofline["step"].update({"nominal_bytes": roofline["step"].pop("bytes"),
                             "nominal_frac": roofline["step"].pop("frac"), "bytes": step_needed,
                             "achieved": round(step_needed / (ms_step * 1e-3) / 1e9, 1),
                             "frac": frac(step_needed, ms_step)})

    cufft = None
    if batch == 1 and not args.no_cufft:
        per_plane = {k: stages[k] / args.steps / planes for k in ("grid", "cols_a", "cols_b")}
        cufft = cufft_compare(torch, wst, plan, work, dev, per_plane, peak)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_img = torch.empty((batch, img_n, img_n), dtype=torch.complex64).pin_memory()
        rows = work.rows_m is not None
        if rows:
            h_rows, h_scale = pin(work.rows_m), pin(work.chan_scale)

        def e2e_step():
            # the C ABI with host buffers: the sort reads the pinned inputs and the last
            # column pass writes the pinned image in place (host <-> device over NVLink-C2C)
            plan.set_vis(h_u, h_v, h_w, h_vis, None, offsets)
            plan.image(out=h_img)

        def rows_step():
            # the same with the inputs as recorded: baseline coordinates per row (metres)
            # and nu / c per channel, expanded to (u, v, w) inside the sort
            plan.set_vis_rows(h_rows, h_scale, h_vis, None, offsets)
            plan.image(out=h_img)

        def copy_step():
            # the same step with explicit copies into device buffers and back
            d_u.copy_(h_u, non_blocking=True)
            d_v.copy_(h_v, non_blocking=True)
            d_w.copy_(h_w, non_blocking=True)
            d_vis.copy_(h_vis, non_blocking=True)
            step()
            h_img.copy_(img, non_blocking=True)

        def timed(fn):
            fn()
            torch.cuda.synchronize(dev)
            n_e2e = max(3, args.steps // 2)
            e0.record(stream)
            for _ in range(n_e2e):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return max_over_ranks(e0.elapsed_time(e1) / n_e2e, dist, dev)

        e2e_ms = timed(e2e_step)
        copy_ms = timed(copy_step)
        d2h = int(8 * batch * img_n * img_n)
        plain = {"value": round(job_mvis(world, n_vis, e2e_ms), 2), "unit": "Mvis/s",
                 "h2d_bytes_per_step": int(20 * n_vis), "d2h_bytes_per_step": d2h,
                 "ms_per_step": round(e2e_ms, 3),
                 "transfer": "host buffers passed to wst_plan_set_vis / wst_image, read and written in place by "
                             "the kernels (pinned memory, NVLink-C2C)"}
        copies = {"value": round(job_mvis(world, n_vis, copy_ms), 2), "ms_per_step": round(copy_ms, 3),
                  "transfer": "wst_plan_set_vis / wst_image on device buffers, cudaMemcpyAsync H2D / D2H around them"}
        if rows:
            rows_ms = timed(rows_step)
            torch.cuda.synchronize(dev)
            # the image of the last end-to-end step against the device-resident step's
            diff = float((h_img.to(dev) - img).abs().max() / img.abs().max())
            e2e = {"value": round(job_mvis(world, n_vis, rows_ms), 2), "unit": "Mvis/s",
                   "h2d_bytes_per_step": int(work.rows_m.nbytes + work.chan_scale.nbytes + 8 * n_vis),
                   "d2h_bytes_per_step": d2h, "ms_per_step": round(rows_ms, 3),
                   "transfer": "host buffers passed to wst_plan_set_vis_rows (baseline metres per row, nu / c "
                               "per channel, values) and wst_image, read and written in place by the kernels "
                               "(pinned memory, NVLink-C2C)",
                   "image_max_diff_rel_peak_vs_device_step": diff,
                   "per_visibility_coordinates": plain, "explicit_copies": copies}
        else:
            e2e = dict(plain, explicit_copies=copies)
        plan.stats()

    # accuracy: the image against the direct transform, with the stated per-pixel bound
    acc = None
    if args.dft_pixels > 0 and batch == 1:
        sigma = kcfg.get("kparam", 0.0)
        acc = accuracy_block(torch, wst, work, st, d_u, d_v, d_w, d_vis, img, dev, args.dft_pixels,
                             args.kernel, cfg.support, sigma, None if table is None else tab_np, args.wfold,
                             osf, plan=plan, n_img=img_n, fov_img=img_fov)
        if not args.snap_w and not args.wfold:
            # the same visibilities with every w moved to its plane's centre: the error
            # against the direct transform is then the (u, v) kernel's alone
            lo, hi = float(st["w_min"]), float(st["w_max"])
            k = torch.clamp(torch.floor((d_w.double() - lo) * (work.n_w / (hi - lo))), 0, work.n_w - 1)
            d_ws = (lo + (k + 0.5) * (hi - lo) / work.n_w).float()
            plan.close()  # its workspace is no longer needed
            plan = wst.Plan(wst.Config(n=img_n, fov=img_fov, n_w=work.n_w, w_min=lo, w_max=hi,
                                       flags=wst.WST_FLAG_KAHAN, planes_per_chunk=min(8, work.n_w),
                                       oversample=args.oversample, grid_n=grid_n, **kcfg), device=dev)
            if table is not None:
                plan.set_kernel_table(table)
            plan.set_vis(d_u, d_v, d_ws, d_vis)
            plan.image(out=img)
            snapped = accuracy_block(torch, wst, work, plan.stats(), d_u, d_v, d_ws, d_vis, img, dev,
                                     args.dft_pixels, args.kernel, cfg.support, sigma,
                                     None if table is None else tab_np, False, osf, plan=plan, n_img=img_n,
                                     fov_img=img_fov)
            acc["w_snapped"] = {k2: snapped[k2] for k2 in (
                "max_err_rel_peak", "central_max_err_rel_peak", "inner3q_max_err_rel_peak",
                "inner3q_rms_err_rel_peak", "max_err_over_bound", "bound_rel_peak", "kernel_error_max")}
            acc["w_snapped"]["what"] = ("every w moved to its plane's centre (same planes, same pixels): the "
                                        "kernel's (u, v) error alone, without the nearest-plane phase error")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and batch == 1:
        job_s, sample, cores, osample, extrap, _ = time_oracle_sample(work, vis_np)
        cpu = {"value": round(n_vis / job_s / 1e6, 4), "unit": "Mvis/s", "cores": cores, "kind": "oracle",
               "sample": sample, "extrapolation": extrap}
        if args.kernel == "gauss" and not args.snap_w and not args.wfold and args.oversample < 2 and not args.image_n:
            cpu["parity_vs_oracle"] = oracle_parity(torch, wst, dev, osample)

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mvis/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n": work.n, "n_w": work.n_w,
                       "n_vis": n_vis, "batch": batch, "kernel": args.kernel, "support": cfg.support, "snap_w": args.snap_w,
                       "table_samples": None if table is None else int(tab_np.size),
                       "wfold": args.wfold, "oversample": round(osf, 4), "image_n": img_n,
                       "grid_n": grid_n or int(round(img_n * osf)),
                       "planes_per_chunk": args.chunk or planes,
                       "n_chunks": st["n_chunks"], "kept": st["n_kept"], "dropped": st["n_dropped"],
                       "rows_gridded": st["n_rows_gridded"],
                       "l2": "inputs larger than L2 (20 B/vis inputs, 8 B/cell planes)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "cufft_compare": cufft,
            "ggpas": {"step": round(n_vis * cfg.support ** 2 / (ms_step * 1e-3) / 1e9, 2),
                      "grid_kernel": round(n_vis * cfg.support ** 2 / (stages["grid"] / args.steps * 1e-3) / 1e9, 2),
                      "note": "grid-point additions per second (N_vis W^2 / time); the grid kernel also "
                              "transforms the rows"},
            "gpu_launches": int(st["n_launches"]) * args.steps, "accuracy": acc,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def run_sharded(args, rank: int, world: int, local_rank: int):
    """One job split over the ranks by w-plane (paper_2301_06061_gb300/shard.py): rank r
    binds the visibilities that the library places in its range of planes, images that
    range (wst_image_range), and the partial images are summed by one all-reduce.  The
    timed step is set_vis + image_range + the all-reduce; value = the job's visibilities
    over the slowest rank's time."""
    import torch

    from paper_2301_06061_gb300 import build, shard, wst

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build.build()
    dev = torch.device("cuda", local_rank)
    work = make_workload(args.workload, 0, args.n_w, args.vis_frac)  # the same job on every rank
    batch = 1 if work.batch_offsets is None else len(work.batch_offsets) - 1
    if batch != 1:
        raise SystemExit("--shard planes images single-image workloads")
    kw = dict(support=work.support, kparam=wst.DEFAULT_SIGMA[work.support])
    d_u, d_v, d_w = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (work.u, work.v, work.w))
    d_vis = torch.empty(work.n_vis, dtype=torch.complex64, device=dev)
    sky_t = [torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
             for a in (work.sky.l, work.sky.m, work.sky.flux)]
    wst.wst_predict_points(d_u, d_v, d_w, *sky_t, d_vis)
    # set-up: the plane of every visibility as the sort assigns it, and the job's w range
    full = wst.Plan(wst.Config(n=work.n, fov=work.fov, n_w=work.n_w, w_min=work.w_min, w_max=work.w_max,
                               flags=wst.WST_FLAG_KAHAN, planes_per_chunk=1, **kw), device=dev)
    full.set_vis(d_u, d_v, d_w, d_vis)
    k = torch.empty(work.n_vis, dtype=torch.int32, device=dev)
    i0, j0 = torch.empty_like(k), torch.empty_like(k)
    wst.wst_vis_cells(full.handle, k, i0, j0)
    st_full = full.stats()
    full.close()
    del i0, j0
    lo, hi = float(st_full["w_min"]), float(st_full["w_max"])
    b, e = shard.plane_ranges(work.n_w, world)[rank]
    own = shard.owned(k, b, e)
    r_u, r_v, r_w, r_vis = d_u[own].contiguous(), d_v[own].contiguous(), d_w[own].contiguous(), d_vis[own].contiguous()
    del k, own
    plan = wst.Plan(wst.Config(n=work.n, fov=work.fov, n_w=work.n_w, w_min=lo, w_max=hi,
                               flags=wst.WST_FLAG_KAHAN | wst.WST_FLAG_TIMING, planes_per_chunk=args.chunk, **kw),
                    device=dev)
    img = torch.empty((1, work.n, work.n), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.set_vis(r_u, r_v, r_w, r_vis)
        plan.image_range(b, e, out=img)
        shard.reduce_images(img, dist)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    plan.stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    st = plan.stats()
    # the reduced image against a single-plan image of the whole job (outside the timed region)
    check = None
    if rank == 0:
        whole = wst.Plan(wst.Config(n=work.n, fov=work.fov, n_w=work.n_w, w_min=lo, w_max=hi,
                                    flags=wst.WST_FLAG_KAHAN, planes_per_chunk=min(8, work.n_w), **kw), device=dev)
        whole.set_vis(d_u, d_v, d_w, d_vis)
        ref = whole.image()
        check = float((img - ref).abs().max() / ref.abs().max())
        whole.close()
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(work.n_vis / (ms_step * 1e-3) / 1e6, 2), "unit": "Mvis/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n": work.n, "n_w": work.n_w,
                       "n_vis": work.n_vis, "parallelism": f"w-plane shards x{world}, one all-reduce of the image",
                       "planes_of_rank0": [b, e], "vis_of_rank0": int(r_u.numel()),
                       "l2": "inputs larger than L2 (20 B/vis inputs, 8 B/cell planes)"},
            "stage_ms_per_step_rank0": {k2: round(st[k2] / args.steps, 4) for k2 in
                                        ("ms_sort", "ms_grid", "ms_cols_a", "ms_cols_b")},
            "reduced_vs_single_plan_max_diff_rel_peak": check, "clocks": clocks,
            "gpu_launches": int(st["n_launches"]) * args.steps, "e2e": None,
            "e2e_note": "the sharded mode times device-resident inputs; the replicas mode reports e2e"}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    work = make_workload(args.workload, 0)
    vis_np = random_values(work, 0)
    if work.batch_offsets is not None:
        print(json.dumps({"impl": "reference", "unavailable": "batched workload: the CPU oracle is timed on "
                          "single-image workloads only"}))
        return
    import oracle

    oracle.build()
    jobs, measured = [], []
    sample = cores = extrap = None
    for i in range(args.warmup + args.steps):
        job_s, sample, cores, _, extrap, step_s = time_oracle_sample(work, vis_np)
        if i >= args.warmup:
            jobs.append(job_s)
            measured.append(step_s)
    job_s = statistics.mean(jobs)
    value = work.n_vis / job_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mvis/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.mean(measured) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n": work.n, "n_w": work.n_w,
                       "n_vis": work.n_vis},
            "step": "one timed sample of the job (gridding of the sample's visibilities, then the sample plane's "
                    "image); ms_per_step is its measured time, value the whole job's throughput extrapolated "
                    "from it (extrapolated_job_ms, extrapolation)",
            "extrapolated_job_ms": round(job_s * 1e3, 1), "extrapolation": extrap,
            "cpu_baseline": {"value": round(value, 4), "unit": "Mvis/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "Mvis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.shard == "planes":
        run_sharded(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
