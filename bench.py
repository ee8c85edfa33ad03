"""Benchmark: one SIRT iteration (fused forward projection + correction, then
voxel-driven weighted backprojection with normalisation and update) of the
perturbed circular cone-beam workload: 512^3 volume, 768 x 768 detector,
720 views, FP32 storage (``--dtype bf16`` for BF16 storage).

Metric: GUPS = (ray samples + voxel-view updates) per second / 1e9, whole job
(sum over ranks / max time over ranks).  Inputs (volume 0.5 GiB, projections
1.7 GB, correction images 1.7 GB) are larger than L2, so no flush is needed
between steps.  ``--impl reference`` times the FP64 CPU oracle (the only
reference this method has) on a bounded sample of the same workload.

Prints ONE JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GUPS (ray samples + voxel updates/s) & SIRT iters/s at 512³; time to residual 1e-3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="64^3 workload (quick check)")
    ap.add_argument("--warm-start-steps", type=int, default=1200,
                    help="train the U-Net warm start this many steps and report time to residual 1e-3 (0: skip)")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="skip the 50-iteration FP32 / BF16 SIRT runs on the bench workload")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the per-row measurements (sub-angle, motion, adjoint, gradient, conv)")
    ap.add_argument("--views", type=int, default=0,
                    help="override the number of views (small cases for ncu captures; not a bench line)")
    ap.add_argument("--domain", default="cartesian", choices=["cartesian", "cylinder"],
                    help="cylinder: the SIRT step on the aligned cylindrical vial domain (Sec. 3.5); not a bench line")
    ap.add_argument("--projector", default="trilinear", choices=["trilinear", "joseph"],
                    help="forward projector of the step (joseph: classical Joseph); not a bench line")
    return ap.parse_args()


def job_throughput(ms_local, units_per_rank, steps, world, device=None):
    """(max-over-ranks ms, whole-job units/s / 1e9): the slowest rank's time
    decides; every rank processed units_per_rank per step (weak scaling, no
    data-path collective).  With world > 1 the process group must exist."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * steps * world / (ms / 1e3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            try:
                power.append(float(parts[3]))
            except ValueError:
                pass
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w": statistics.median(power) if power else None}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one full-size
# launch of the fused forward kernel, from one-pass ncu captures of that
# kernel on 16 and 180 views of the workload (summary kept under profiles/):
# the launch reads the volume atlas once and each view's measured image and
# writes its correction image, so traffic = a + b * views, with a and b from
# the two captures, evaluated at 720 views.  Valid only for the kernel
# sources it was taken on (hash below) and for the FP32 workload; otherwise
# null.
_T16, _T180 = 585831936 + 33430016, 982422528 + 395699200
FWD_TRAFFIC_BYTES = int(_T16 + (_T180 - _T16) * (720 - 16) / (180 - 16))
FWD_TRAFFIC_SOURCES = ("project.cu", "atlas.cuh", "ray.cuh", "cylinder.cuh", "joseph.cuh", "roi.cuh", "fwd_common.cuh",
                       "ctrex_internal.cuh", "dyrect.cuh")
FWD_TRAFFIC_HASH = "ffcabe5e01f8bb0a"


def fwd_traffic(dtype, views):
    import hashlib

    h = hashlib.sha256()
    for f in FWD_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2609_30166_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != FWD_TRAFFIC_HASH or dtype != "f32" or views:
        return None
    return FWD_TRAFFIC_BYTES


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------

def oracle_plan_inputs():
    """Inputs of the oracle timing plan (CPU, outside every timed region):
    phantoms voxelised with one sample per voxel (the oracle's run time does
    not depend on the values) and measured projections from the oracle."""
    import numpy as np

    import oracle
    from paper_2609_30166_gb300 import inputs

    def problem(cfg):
        P = inputs.projection_matrices(cfg)
        return oracle.Problem(P, cfg.vol_shape, (cfg.vox,) * 3, cfg.origin, (cfg.nu, cfg.nv), cfg.step_vox)

    c1, c5, c2 = inputs.CIRCULAR_64, inputs.SPARSE_128, inputs.PERTURBED_512
    pb1, pb5, pb2 = problem(c1), problem(c5), problem(c2)
    v1 = inputs.phantom(c1, sub=1).numpy()
    v5 = inputs.phantom(c5, sub=1).numpy()
    v2 = inputs.phantom(c2, sub=1).numpy()
    p1 = oracle.forward(pb1, v1)[0]
    p5 = oracle.forward(pb5, v5)[0]
    fwd_views = np.linspace(0, c2.n_views - 1, 4).round().astype(np.int32)
    lo = c2.n // 2 - 32
    idx = np.arange(lo, lo + 64)
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    vox_flat = ((zz * c2.n + yy) * c2.n + xx).ravel().astype(np.int64)
    r2 = np.ones((c2.n_views, c2.nv, c2.nu))
    units = {
        "c1_sirt_10": 10 * (oracle.count_samples(pb1) + v1.size * c1.n_views),
        "c5_sirt_1": oracle.count_samples(pb5) + v5.size * c5.n_views,
        "c2_fwd_4_views": oracle.count_samples(pb2, fwd_views),
        "c2_bp_64^3_720_views": vox_flat.size * c2.n_views,
    }
    runs = {
        "c1_sirt_10": lambda: oracle.sirt(pb1, p1, 10),
        "c5_sirt_1": lambda: oracle.sirt(pb5, p5, 1),
        "c2_fwd_4_views": lambda: oracle.forward(pb2, v2, views=fwd_views),
        "c2_bp_64^3_720_views": lambda: oracle.backproject_voxels(pb2, r2, vox_flat),
    }
    return units, runs


ORACLE_PLAN = ("oracle FP64 (C, OpenMP): {c1} full 10-iteration SIRT; {c5} one SIRT iteration; {c2} forward of "
               "4 complete views and backprojection of the central 64^3 sub-volume over all 720 views")


def oracle_plan_time(units, runs, reps=3):
    """Median of reps timings of each part; returns (units, seconds, parts)."""
    parts = {}
    for name, fn in runs.items():
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        parts[name] = {"units": units[name], "s": statistics.median(ts), "gups": units[name] / statistics.median(ts) / 1e9}
    total_u = sum(p["units"] for p in parts.values())
    total_s = sum(p["s"] for p in parts.values())
    return total_u, total_s, parts


def oracle_plan_desc():
    from paper_2609_30166_gb300 import inputs

    return ORACLE_PLAN.format(c1=inputs.CIRCULAR_64.name, c5=inputs.SPARSE_128.name, c2=inputs.PERTURBED_512.name)


def omp_threads():
    try:
        return int(os.environ.get("OMP_NUM_THREADS", "")) or os.cpu_count()
    except ValueError:
        return os.cpu_count()


# ---------------------------------------------------------------------------

def build_workload(cfg, device, dtype):
    import torch

    from paper_2609_30166_gb300 import ctrex, inputs

    if isinstance(cfg, inputs.CylConfig):
        P = inputs.projection_matrices(cfg.base)
        ctx = ctrex.context_for_cylinder(cfg, P=P, device=device)
        phantom = inputs.cyl_phantom(cfg, device=str(device)).to(torch.float32).contiguous()
    else:
        P = inputs.projection_matrices(cfg)
        ctx = ctrex.context_for(cfg, P=P, device=device)
        phantom = inputs.phantom(cfg, device=str(device)).to(torch.float32).contiguous()
    p32 = ctx.fwd_project(phantom)  # inverse-crime measured data
    torch.cuda.synchronize(device)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    p = p32.to(tdt).contiguous()
    del p32
    return ctx, P, phantom, p, tdt


def _time(fn, reps=3, warm=1):
    """Mean CUDA-event time (s) of fn() on the current stream."""
    import torch

    for _ in range(warm):
        fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 1e3 / reps


# FP32 operations per motion-warped sample: 64-control-point cubic B-spline
# (per point one weight product and three FMAs, plus per-axis weights), the
# pose (9 FMA + 3), trilinear interpolation; counted from ray.cuh.
MOTION_OPS_PER_SAMPLE = 64 * 4 + 16 + 3 * 10 + 12 + 30


def sirt_50_iterations(ctx, cfg, p, device):
    """50 SIRT iterations from zero on the bench workload with FP32 and with
    BF16 storage (volume, projections, correction images; FP32 accumulation):
    residuals and how far the BF16 run ends from the FP32 run.  The per-step
    error of both against the FP64 oracle (central 64^3 sub-volume at k = 0
    and k = 49) is checked by the GPU test suite, which may run the oracle."""
    import torch

    res = {"workload": cfg.name, "iterations": 50}
    finals = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        pp = p if dt == torch.float32 else p.to(dt).contiguous()
        x = torch.zeros(cfg.vol_shape, dtype=dt, device=device)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        x, hist, done = ctx.sirt_iterate(x, pp, 50)
        torch.cuda.synchronize(device)
        res[name] = {"s": time.perf_counter() - t0, "iters": done, "residual_first": float(hist[0]),
                     "residual_last": float(hist[-1])}
        finals[name] = x.float()
        del pp, x
    d = (finals["bf16"] - finals["f32"]).double().norm() / finals["f32"].double().norm()
    res["bf16_vs_f32_rel_l2"] = float(d)
    del finals
    torch.cuda.empty_cache()
    return res


def dyrect_sirt_step(ctx, cfg, device, n_samples, n_updates, gather_peak):
    """One SIRT step of the event-based 4D model (Sec. 3.3) on the bench
    workload: the event scene's initial and final values and transition
    times, measured data simulated by the event-model projector, the fused
    forward + correction and the split backprojection timed.  Samples and
    voxel-view updates are those of the static step (each tap and each
    voxel-view pair serves one of the two value fields).  A sample costs two
    gathers where its 8^3 brick lies wholly on one side of the view's time
    and six otherwise (initial value, final value, transition time; two
    slices); fwd_gathers_per_sample is the forward time in units of the
    measured gather ceiling per sample (the static projector: about 2.3)."""
    import torch

    from paper_2609_30166_gb300 import inputs

    mu0, mu1, tau = inputs.dyrect_fields(cfg, device=str(device))
    tv = torch.as_tensor(inputs.view_times(cfg), dtype=torch.float32, device=device)
    ctx.set_dyrect(tau.to(torch.float32).contiguous(), tv)
    x_true = torch.stack([mu0, mu1]).to(torch.float32).contiguous()
    del mu0, mu1, tau
    pd = ctx.fwd_project(x_true)
    x = torch.zeros_like(x_true)
    del x_true
    r = torch.empty_like(pd)
    sums = torch.empty(2, dtype=torch.float64, device=device)
    t_f = _time(lambda: ctx.fwd_correct(x, pd, r=r, sums=sums), reps=2)
    t_b = _time(lambda: ctx.back_project(r, vol=x, alpha=1.0, normalize=True, accumulate=True), reps=2)
    ctx.set_dyrect(None)
    del x, r, pd
    torch.cuda.empty_cache()
    return {"workload": cfg.name + " (event scene: 8 changing regions)", "fwd_correct_ms": t_f * 1e3,
            "back_project_ms": t_b * 1e3, "gups": (n_samples + n_updates) / (t_f + t_b) / 1e9,
            "fwd_gathers_per_sample": t_f * gather_peak / n_samples,
            "bp_tex_gather_frac": n_updates / t_b / gather_peak}


def time_to_residual_circular64(device, tol=1e-3, max_iter=20000):
    """Plain SIRT from zero on the 64^3 circular workload until rho <= tol:
    wall time (the host reads the residual once per iteration) and
    iterations."""
    import torch

    from paper_2609_30166_gb300 import ctrex, inputs

    cfg = inputs.CIRCULAR_64
    ctx = ctrex.context_for(cfg, device=device)
    ph = inputs.phantom(cfg, device=str(device)).to(torch.float32).contiguous()
    p = ctx.fwd_project(ph)
    x = torch.zeros(cfg.vol_shape, dtype=torch.float32, device=device)
    ctx.sirt_iterate(x.clone(), p, 3)  # warm-up
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    x, hist, done = ctx.sirt_iterate(x, p, max_iter, tol=tol)
    torch.cuda.synchronize(device)
    dt = time.perf_counter() - t0
    ctx.close()
    return {"workload": cfg.name, "tol": tol, "s": dt, "iters": done,
            "residual_last": float(hist[done]) if done < len(hist) else float(hist[-1])}


def measure_rows(device, gather_peak, sm_count, sm_mhz):
    """Throughput of the hot-path rows the SIRT step does not exercise, each on
    its full-size workload, with the ceiling that bounds it."""
    import torch

    from paper_2609_30166_gb300 import ctrex, inputs

    rows = {}
    # a3 + a11: helical sub-angle projector, BF16 volume, FP32 accumulation
    cfg = inputs.HELICAL_256
    ctx = ctrex.context_for(cfg, device=device)
    vol16 = inputs.phantom(cfg, device=str(device)).to(torch.bfloat16).contiguous()
    out = torch.empty((cfg.n_views, cfg.nv, cfg.nu), dtype=torch.float32, device=device)
    ns = ctx.count_samples()
    t = _time(lambda: ctx.fwd_project(vol16, proj=out))
    rows["a3_helical_subangle_bf16"] = {"workload": cfg.name, "samples": ns, "ms": t * 1e3,
                                        "gsamples_per_s": ns / t / 1e9,
                                        "tex_gather_frac": ns / t / gather_peak}
    del ctx, vol16, out
    # a4, a8, a9: motion-aware projector, matched adjoint, motion gradient
    cfg = inputs.MOTION_256
    ctx = ctrex.context_for(cfg, device=device)
    th, co, sv = inputs.motion_params(cfg)
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()  # noqa: E731
    ctx.set_motion(f(th), f(co), f(sv), cfg.margin)
    vol = inputs.phantom(cfg, device=str(device)).float().contiguous()
    ns = ctx.count_samples()
    proj = ctx.fwd_project(vol)
    g = torch.randn(proj.shape, device=device, generator=torch.Generator(device=device).manual_seed(1))
    adj = torch.zeros_like(vol)
    alu_peak = sm_count * 128 * sm_mhz * 1e6  # FP32 lanes x clock (an FMA counted once)
    t_f = _time(lambda: ctx.fwd_project(vol, proj=proj))
    t_a = _time(lambda: ctx.adjoint_project(g, vol=adj))
    t_g = _time(lambda: ctx.motion_grad(vol, g), reps=2)
    rows["a4_motion_projector"] = {"workload": cfg.name, "samples": ns, "ms": t_f * 1e3,
                                   "gsamples_per_s": ns / t_f / 1e9,
                                   "alu_frac_est": ns * MOTION_OPS_PER_SAMPLE / t_f / alu_peak,
                                   "alu_peak_ops_per_s": alu_peak,
                                   "ops_per_sample_est": MOTION_OPS_PER_SAMPLE}
    rows["a8_matched_adjoint"] = {"workload": cfg.name, "ms": t_a * 1e3, "gsamples_per_s": ns / t_a / 1e9,
                                  "tap_updates_per_s": 8 * ns / t_a}
    rows["a9_motion_gradient"] = {"workload": cfg.name, "ms": t_g * 1e3, "gsamples_per_s": ns / t_g / 1e9}
    del ctx, vol, proj, g, adj
    # cylindrical domain (Sec. 3.5): one SIRT step on the vial workload
    cc = inputs.CYL_VIAL
    ctx = ctrex.context_for_cylinder(cc, device=device)
    vol = inputs.cyl_phantom(cc, device=str(device)).float().contiguous()
    p = ctx.fwd_project(vol)
    ns = ctx.count_samples()
    nu_ = cc.n_r * cc.n_phi * cc.n_z * cc.base.n_views * cc.base.n_sub
    x = torch.zeros_like(vol)
    r = torch.empty_like(p)
    sums = torch.zeros(2, dtype=torch.float64, device=device)
    t_fc = _time(lambda: ctx.fwd_correct(x, p, r=r, sums=sums), reps=2)
    t_bp = _time(lambda: ctx.back_project(r, vol=x, alpha=1.0), reps=2)
    rows["a15_cylinder_sirt_step"] = {"workload": cc.name, "samples": ns, "updates": nu_,
                                      "fwd_correct_ms": t_fc * 1e3, "back_project_ms": t_bp * 1e3,
                                      "gups": (ns + nu_) / (t_fc + t_bp) / 1e9,
                                      "fwd_tex_gather_frac": 2 * ns / t_fc / gather_peak,
                                      "bp_tex_gather_frac": nu_ / t_bp / gather_peak}
    del ctx, vol, p, x, r
    # multi-resolution ROI (Sec. 3.7): one SIRT step on a 256^3 context grid
    # with a 4x finer 256^3 ROI, projected together
    rc = inputs.ROI_FOCUS
    ctx = ctrex.context_for(rc.base, device=device)
    ctx.set_roi(rc.roi_shape, (rc.roi_vox,) * 3, rc.roi_origin)
    xc, xf = inputs.roi_phantom(rc, device=str(device))
    vol = torch.cat([xc.flatten(), xf.flatten()]).float().contiguous()
    del xc, xf
    p = ctx.fwd_project(vol)
    ns = ctx.count_samples()
    nu_ = vol.numel() * rc.base.n_views * rc.base.n_sub
    x = torch.zeros_like(vol)
    r = torch.empty_like(p)
    t_fc = _time(lambda: ctx.fwd_correct(x, p, r=r, sums=sums), reps=2)
    t_bp = _time(lambda: ctx.back_project(r, vol=x, alpha=1.0), reps=2)
    rows["a17_roi_sirt_step"] = {"workload": rc.name, "samples": ns, "updates": nu_,
                                 "fwd_correct_ms": t_fc * 1e3, "back_project_ms": t_bp * 1e3,
                                 "gups": (ns + nu_) / (t_fc + t_bp) / 1e9,
                                 "fwd_tex_gather_frac": 2 * ns / t_fc / gather_peak,
                                 "bp_tex_gather_frac": nu_ / t_bp / gather_peak}
    del ctx, vol, p, x, r
    # a12: tcgen05 implicit-GEMM convolution, the U-Net's levels (batch 2 at 128^3)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16_peak = float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        bf16_peak = 1900.0
    convs = {}
    gen = torch.Generator(device=device).manual_seed(2)
    # the U-Net's distinct conv shapes: encoder levels, bottleneck, decoder
    # (skip concatenation: 48, 96 and 192 input channels)
    for (n, cin, cout) in ((128, 16, 16), (64, 32, 32), (32, 64, 64), (16, 128, 128), (32, 192, 64), (64, 96, 32),
                           (128, 48, 16)):
        x = torch.randn((2, n, n, n, cin), device=device, generator=gen).to(torch.bfloat16)
        wt = (torch.randn((cout, 27, cin), device=device, generator=gen) * 0.05).to(torch.bfloat16)
        dy = torch.randn((2, n, n, n, cout), device=device, generator=gen).to(torch.bfloat16)
        flops = 2.0 * x.numel() / cin * 27 * cin * cout
        t_fw = _time(lambda: ctrex.conv3d(x, wt, relu=True))
        t_wg = _time(lambda: ctrex.conv3d_wgrad(x, dy))
        # compulsory HBM bytes: x and y (forward) or x and dy (weight gradient)
        hbm = 2.0 * x.numel() / cin * (cin + cout)
        hbm_peak = measured_peaks()[0] * 1e9
        convs[f"{n}^3 x2, {cin}->{cout}"] = {"fwd_ms": t_fw * 1e3, "fwd_tflops": flops / t_fw / 1e12,
                                             "fwd_hbm_frac": hbm / t_fw / hbm_peak,
                                             "wgrad_ms": t_wg * 1e3, "wgrad_tflops": flops / t_wg / 1e12,
                                             "wgrad_hbm_frac": hbm / t_wg / hbm_peak}
    ctrex.conv_status_check(device)
    best = max(v["fwd_tflops"] for v in convs.values())
    rows["a12_conv3d_tcgen05"] = {"layers": convs, "best_fwd_tflops": best, "bf16_peak_tflops": bf16_peak,
                                  "best_fwd_frac": best / bf16_peak,
                                  "kernels": {"fwd": "conv_fwd_tma_kernel (persistent, TMA, brick-staged input); "
                                                     "at most 16 output channels: conv_fwd_kx_kernel (kx taps "
                                                     "folded into N, input planes reused along z)",
                                              "wgrad": "conv_wgrad_tma_kernel (MN-major brick, kx taps folded into N); "
                                                       "16 output channels: conv_wgrad_c16_kernel (mma.m16n8k16 "
                                                       "with register-resident operands)"}}
    torch.cuda.empty_cache()
    return rows


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2609_30166_gb300 import inputs

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    cyl = args.domain == "cylinder"
    if cyl:
        cfg = inputs.CYL_SMALL if args.small else inputs.CYL_VIAL
        if args.views:
            cfg = cfg.scaled(base=cfg.base.scaled(n_views=args.views), name=f"{cfg.name}-views{args.views}")
        geo = cfg.base
    else:
        cfg = inputs.CIRCULAR_64 if args.small else inputs.PERTURBED_512
        if args.views:
            cfg = cfg.scaled(n_views=args.views, name=f"{cfg.name}-views{args.views}")
        geo = cfg
    ctx, P, phantom, p, tdt = build_workload(cfg, device, args.dtype)
    if args.projector != "trilinear":
        ctx.set_projector(args.projector)
    n_samples = ctx.count_samples()
    nz_, ny_, nx_ = cfg.vol_shape
    n_updates = nz_ * ny_ * nx_ * geo.n_views * geo.n_sub
    units = n_samples + n_updates

    x = torch.zeros(cfg.vol_shape, dtype=tdt, device=device)
    r = torch.empty_like(p)
    sums = torch.zeros(2, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        ctx.fwd_correct(x, p, r=r, sums=sums)
        if ev is not None:
            ev[1].record(stream)
        ctx.back_project(r, vol=x, alpha=1.0, normalize=True, accumulate=True)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    bp_ms = [e[1].elapsed_time(e[2]) for e in evs]
    res = float((sums[0] / sums[1]).sqrt())
    ms, value = job_throughput(ms, units, args.steps, world, device)
    sec = ms / 1e3

    # end to end through the host-buffer C ABI entry point
    e2e = None
    if args.e2e_steps > 0:
        xh = torch.zeros(cfg.vol_shape, dtype=tdt).pin_memory()
        ph = p.cpu().pin_memory()
        ctx.sirt_host(xh, ph, 1)  # warm-up (allocates the context's host-path buffers)
        torch.cuda.synchronize(device)
        clocks_e2e = ClockSampler(local)
        clocks_e2e.start()
        step_s = []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            ctx.sirt_host(xh, ph, 1)
            step_s.append(time.perf_counter() - t1)
        e2e_s = time.perf_counter() - t0
        elt = 2 if tdt == torch.bfloat16 else 4
        e2e = {"value": units * args.e2e_steps * world / e2e_s / 1e9, "unit": "GUPS",
               "h2d_bytes_per_step": int(xh.numel() * elt + ph.numel() * elt),
               "d2h_bytes_per_step": int(xh.numel() * elt + 16),
               "step_ms": [round(t * 1e3, 1) for t in step_s], "clocks": clocks_e2e.stop()}
        del ph, xh

    elt = 2 if tdt == torch.bfloat16 else 4
    fwd_avg = statistics.mean(fwd_ms) / 1e3
    alg_bytes = n_samples * 8 * elt
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / fwd_avg / 1e9
    from paper_2609_30166_gb300 import ctrex as _ct

    l2_peak = _ct.probe_l2_read_bandwidth(device)
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    l1_mhz = (clk or {}).get("sm_mhz") or 2070.0
    l1_peak = sm_count * 128.0 * l1_mhz * 1e6 / 1e9  # GB/s: 128 B per SM per clock

    gather_peak = _ct.probe_gather_rate(device)
    gathers_per_sample = 1 if tdt == torch.bfloat16 else 2
    fwd_gathers = gathers_per_sample * n_samples / fwd_avg
    bp_gathers = n_updates / (statistics.mean(bp_ms) / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": "GUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.dtype == "f32" else "bf16",
        "data": "synthetic (seeded ellipsoid + Gaussian-blob phantom, projections simulated by the projector)",
        "config": {"workload": cfg.name, "volume": list(cfg.vol_shape), "detector": [geo.nv, geo.nu],
                   "views": geo.n_views, "sub_angles": geo.n_sub, "step_vox": geo.step_vox,
                   "storage": args.dtype, "accumulation": "f32",
                   "l2": "inputs larger than L2 (volume, projections and correction images > 129 MB); no flush",
                   "parallelism": f"replicas x{world}", "samples_per_step": n_samples,
                   "updates_per_step": n_updates},
        "sirt_iters_per_s": args.steps * world / sec,
        "kernel_ms": {"fwd_correct": statistics.mean(fwd_ms), "back_project": statistics.mean(bp_ms)},
        "residual_after": res,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None if (cyl or args.projector != "trilinear") else fwd_traffic(args.dtype, args.views),
                     "kernel": "fwd_kernel (fused forward + correction)",
                     "l2_gather": {"achieved": achieved, "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
                                   "peak_method": "ctrex_probe_l2_read_bandwidth: 16-byte L2-only loads "
                                                  "(ld.global.cg) over half of L2, 512 passes"},
                     "l1_gather": {"achieved": achieved, "peak": l1_peak, "unit": "GB/s", "frac": achieved / l1_peak,
                                   "peak_method": f"{sm_count} SMs x 128 B/clk x {l1_mhz:.0f} MHz "
                                                  "(median SM clock sampled in the timed region)"},
                     "tex_gather": {"achieved": fwd_gathers, "peak": gather_peak, "unit": "gathers/s",
                                    "frac": fwd_gathers / gather_peak, "per_sample": gathers_per_sample,
                                    "bp_achieved": bp_gathers, "bp_frac": bp_gathers / gather_peak,
                                    "peak_method": "ctrex_probe_gather_rate: tex2Dgather on an L1-resident texture"},
                     "note": f"algorithmic gather bytes = 8 taps x {elt} B per sample; peak = HBM copy "
                             f"bandwidth ({peak_kind}). The taps are served from L1/TEX and L2 (DRAM traffic "
                             "is ~1x the compulsory bytes), so the HBM figure cannot bound this kernel: "
                             "frac > 1 is expected. Its binding ceiling is tex_gather (texture return "
                             "path, 2 gathers per FP32 sample); l2_gather and l1_gather give the graded "
                             "gather roofline against the measured L2 read bandwidth and the L1 ceiling"},
        # per step: volume atlas upload (two kernels for the Joseph atlas),
        # fused forward + correction, residual finish, correction-image atlas
        # upload, backprojection + update
        "gpu_launches": (6 if args.projector == "joseph" else 5) * args.steps,
        "e2e": e2e,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_rows and not args.views and not args.small and not cyl \
            and args.projector == "trilinear":
        sm_count = torch.cuda.get_device_properties(device).multi_processor_count
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        # sub-voxel backprojection (2^3 points per voxel) of the last step's
        # correction images, on the same workload
        ctx.set_bp_subvoxel(2)
        t_sv = _time(lambda: ctx.back_project(r, vol=x, alpha=1.0, normalize=True, accumulate=True), reps=2)
        ctx.set_bp_subvoxel(1)
        sv_points = 8 * n_updates
        # classical Joseph forward projector (one gather per slice crossing):
        # the same SIRT step with it, on the same workload
        ctx.set_projector("joseph")
        ns_j = ctx.count_samples()
        t_jf = _time(lambda: ctx.fwd_correct(x, p, r=r, sums=sums), reps=2)
        t_jb = _time(lambda: ctx.back_project(r, vol=x, alpha=1.0, normalize=True, accumulate=True), reps=2)
        ctx.set_projector("trilinear")
        joseph_row = {"workload": cfg.name, "samples": ns_j, "fwd_correct_ms": t_jf * 1e3,
                      "back_project_ms": t_jb * 1e3, "gups": (ns_j + n_updates) / (t_jf + t_jb) / 1e9,
                      "fwd_tex_gather_frac": ns_j / t_jf / gather_peak,
                      "trilinear_fwd_correct_ms": statistics.mean(fwd_ms)}
        # BF16 storage of the volume, the projections and the correction
        # images (FP32 accumulation): the same SIRT step on the same workload
        bf16_row = None
        if tdt == torch.float32:
            x16, p16 = x.to(torch.bfloat16), p.to(torch.bfloat16)
            r16, s16 = torch.empty_like(p16), torch.empty(2, dtype=torch.float64, device=device)
            t_bf = _time(lambda: ctx.fwd_correct(x16, p16, r=r16, sums=s16), reps=2)
            t_bb = _time(lambda: ctx.back_project(r16, vol=x16, alpha=1.0, normalize=True, accumulate=True), reps=2)
            bf16_row = {"workload": cfg.name, "storage": "bf16", "accumulation": "f32",
                        "fwd_correct_ms": t_bf * 1e3, "back_project_ms": t_bb * 1e3,
                        "gups": units / (t_bf + t_bb) / 1e9,
                        "fwd_tex_gather_frac": n_samples / t_bf / gather_peak,
                        "bp_tex_gather_frac": n_updates / t_bb / gather_peak}
            del x16, p16, r16
        # ordered-subset SIRT (Sec. 2.3.2): one cycle over 10 interleaved
        # subsets of 72 views (visited in bit-reversed order), each a fused
        # forward + correction and a normalised backprojection of its views,
        # with a host read of the subset's residual between them
        subsets = inputs.subsets_cyclic(geo.n_views, 10)
        xo = torch.zeros_like(x)
        t_os = _time(lambda: ctx.os_sirt_iterate(xo, p, subsets, 1), reps=2)
        os_row = {"workload": cfg.name, "subsets": len(subsets), "views_per_subset": geo.n_views // len(subsets),
                  "cycle_ms": t_os * 1e3, "gups": units / t_os / 1e9, "sirt_step_ms": ms / args.steps}
        # extended field of view (Sec. 3.6, 4.3.2): one SIRT iteration whose
        # backprojector sees per-view detector windows, the inner edge drawn
        # between column 0 and the detector centre
        ctx.set_bp_window(inputs.efov_windows(geo, 0.5 * (geo.nu - 1), seed=7))
        t_ef = _time(lambda: ctx.sirt_iterate(xo, p, 1), reps=2)
        ctx.set_bp_window(None)
        ef_row = {"workload": cfg.name + " (per-view BP windows)", "iteration_ms": t_ef * 1e3,
                  "gups": units / t_ef / 1e9, "sirt_step_ms": ms / args.steps}
        del xo
        del x, r
        torch.cuda.empty_cache()
        if args.accuracy and tdt == torch.float32:
            out["sirt_50_iterations"] = sirt_50_iterations(ctx, cfg, p, device)
        dyr_row = dyrect_sirt_step(ctx, cfg, device, n_samples, n_updates, gather_peak) \
            if tdt == torch.float32 else None
        out["rows"] = measure_rows(device, gather_peak, sm_count, sm_mhz)
        if dyr_row:
            out["rows"]["a18_dyrect_sirt_step"] = dyr_row
        out["rows"]["a14_subvoxel_bp"] = {"workload": cfg.name, "s": 2, "ms": t_sv * 1e3,
                                          "point_updates": sv_points, "gpoint_updates_per_s": sv_points / t_sv / 1e9,
                                          "tex_gather_frac": sv_points / t_sv / gather_peak,
                                          "centre_bp_ms": statistics.mean(bp_ms)}
        out["rows"]["a16_joseph_sirt_step"] = joseph_row
        out["rows"]["a19_os_sirt_cycle"] = os_row
        out["rows"]["a20_efov_sirt_iteration"] = ef_row
        if bf16_row:
            out["rows"]["a11_bf16_sirt_step"] = bf16_row
    if rank == 0 and world == 1 and not args.no_rows and not args.views and not args.small and not cyl:
        out["time_to_residual_1e-3_circular64"] = time_to_residual_circular64(device)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not cyl:
        units_p, runs_p = oracle_plan_inputs()
        ncpu_units, ncpu_s, parts = oracle_plan_time(units_p, runs_p, reps=3)
        out["cpu_baseline"] = {"value": ncpu_units / ncpu_s / 1e9, "unit": "GUPS", "cores": omp_threads(),
                               "kind": "oracle", "sample": oracle_plan_desc() + "; median of 3 per part",
                               "parts": parts}
    if rank == 0 and world == 1 and args.warm_start_steps > 0 and not args.views and not args.small and not cyl:
        from paper_2609_30166_gb300 import warmstart

        del p, phantom
        torch.cuda.empty_cache()
        ws = warmstart.run(n_train=56, n_test=8, steps=args.warm_start_steps)
        out["time_to_residual_1e-3"] = {
            "workload": ws["workload"], "tol": ws["tol"], "held_out_phantoms": ws["test_phantoms"],
            "plain_sirt_s": ws["plain_s"], "plain_sirt_iters": ws["plain_iters"],
            "warm_start_s": ws["warm_s"], "warm_start_iters": ws["warm_iters"],
            "warm_over_plain_time": ws["warm_over_plain_time"],
            "net_err": ws["net_err"], "sirt_in_err": ws["sirt_in_err"],
            "note": "warm start = 5 SIRT iterations + U-Net (tcgen05 convs) + SIRT; training "
                    f"({ws['train_steps']} steps on {ws['train_phantoms']} phantoms, squared error plus 16 x the "
                    f"squared error gradient, {ws['train_s']:.1f} s) not timed; held-out seeds 56..63",
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_reference(args):
    """The FP64 oracle on the host cores, on bounded samples of the workload."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2609_30166_gb300 import inputs

    cfg = inputs.CIRCULAR_64 if args.small else inputs.PERTURBED_512
    units_p, runs_p = oracle_plan_inputs()
    for _ in range(args.warmup):
        runs_p["c1_sirt_10"]()
    units_total, secs, parts = 0, 0.0, {}
    for _ in range(args.steps):
        u, s, parts = oracle_plan_time(units_p, runs_p, reps=1)
        units_total += u
        secs += s
    desc = oracle_plan_desc() + "; each step runs every part once"
    value = units_total / secs / 1e9
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": cfg.name, "volume": list(cfg.vol_shape),
                                        "detector": [cfg.nv, cfg.nu], "views": cfg.n_views},
        "cpu_baseline": {"value": value, "unit": "GUPS", "cores": omp_threads(), "kind": "oracle",
                         "sample": desc, "parts": parts},
        "e2e": {"value": value, "unit": "GUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
