#!/usr/bin/env python
"""Benchmark of the Blacklight hot path on GB300: rays/s of geodesic + polarized transfer.

Workload (one step): 9 images -- spins {0, 0.5, 0.94} x inclinations {17, 60, 90} deg -- of
256x256 pixels each, camera at r = 1000 M with a +-20 M field of view, 230 GHz, on the seeded
synthetic torus sampled on a 256x128x128 spherical Kerr-Schild grid (one grid per spin), traced
in one batched persistent launch pair. Inputs stay resident in HBM; the three grids (3 x 134 MB)
plus the per-sample records exceed the 129 MB L2, so no explicit flush is needed between steps.

One JSON line is printed by rank 0. See the design notes for the roofline arithmetic.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/sec (geodesic+polarized transfer) at 256^2"
SPINS = (0.0, 0.5, 0.94)
INCS = (17.0, 60.0, 90.0)
FREQ = 230e9
N_PIX = 256
GRID = (256, 128, 128)
# Algorithmic arithmetic per unit of work (operation counts of the method, see design notes):
# FP64 flops per Dormand-Prince attempt: 6 right-hand sides of 114 flops (81 products, 30
# sums, 2 reciprocal square roots, 1 reciprocal in the form with d_c(l.k) taken directly),
# 6 stage combinations (384), the embedded error estimate (96) and its norm and the step
# control (50).
FLOP64_PER_ATTEMPT = 1214
# dram__bytes_read.sum + dram__bytes_write.sum of geodesic_kernel<float, df64> per DP attempt
# from one ncu capture of the a = 0.94, i = 60 deg image of this workload at 256^2; None
# whenever the kernel has changed since the capture (the last capture, 147.7 B, predates the
# interleaved ray queue of image batches)
GEO_DF64_DRAM_BYTES_PER_ATTEMPT = None
# FP32 flops per transfer sample (2 transport matrices, predictor-corrector, sampling,
# plasma, coefficients, fluid frame, Stokes step)
FLOP32_PER_SAMPLE = 3300
# Nominal peaks from the pool's profiling recipe (no measured FP64/FP32 peak is available):
# FP64 1.25 TFLOP/s; FP32 = 152 SMs x 128 lanes x 2 flop x 2.07 GHz.
PEAK_FP64_TFLOPS = 1.25
# Double-float: FP32 instructions per emulated FP64 flop as implemented -- a product 7 (4 inside
# a chain of products), a sum 11, a scaling by a power of two 2, a reciprocal ~9 and a
# reciprocal square root ~12 (hardware seed and one second-order step), a term of a
# compensated sum of products 12 (first product 4, a plain term 7, the final renormalisation
# 3, y + h sum 15), an FP32 flop 1. On the attempt's mix (right-hand sides 719 instructions for
# 114 flops, stage combinations 2352 for 384, error estimate 576 for 96, norm and control ~60
# for 50) that is 7302 instructions for 1214 flops, 6.0 per flop. The emulated peak is the
# FP32 issue rate (152 SMs x 128 lanes x 2.07 GHz instructions/s) divided by that.
DF64_INSTR_PER_FLOP = 6.0
PEAK_DF64_TFLOPS = 152 * 128 * 2.07e9 / DF64_INSTR_PER_FLOP / 1e12
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="blacklight", choices=["blacklight", "reference"])
    ap.add_argument("--precision", default="fast", choices=["mixed", "fp64", "fast"],
                    help="fast: double-float geodesics + FP32 transfer (default); mixed: FP64 "
                         "geodesics + FP32 transfer; fp64: FP64 throughout")
    ap.add_argument("--no-other-forms", action="store_true",
                    help="skip the short timing of the two other precision forms")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: one 256^2 image (a=0.94, i=60 deg) of the same workload, for "
                         "profiler captures")
    ap.add_argument("--grid-layout", default="cells", choices=["cells", "planes"],
                    help="memory order of the device grids: cells (repacked once by "
                         "blacklight_grid_pack) or planes (as generated)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-hires", action="store_true",
                    help="skip the 1024^2 image on the 512x256x256 torus")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the batched adaptive-refinement workload")
    ap.add_argument("--coef", default="exact", choices=["exact", "mlp"],
                    help="coefficients of the main workload: exact fits, or the learned model "
                         "(trained first; needs --precision fast or mixed)")
    ap.add_argument("--no-slow", action="store_true",
                    help="skip the slow-light line (8 snapshots, 512^2)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the unpolarized, auxiliary-image and RK4/RK2 timings")
    ap.add_argument("--no-plan", action="store_true",
                    help="skip the autotuned CUDA-graph plan line")
    ap.add_argument("--no-mlp", action="store_true",
                    help="skip the learned-coefficient line (training + 1024^2 image + FP64 form)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_elapsed(torch, elapsed, world, device):
    """Slowest rank's timed-region length (ranks trace independent replicas, no exchange)."""
    if world <= 1:
        return elapsed
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, rays_per_rank_step, steps, elapsed_max):
    """Whole-job rays/s: every rank's rays over the slowest rank's time."""
    return world * rays_per_rank_step * steps / elapsed_max


# memory order of the device grids the bench traces ("cells" or "planes"; set from --grid-layout)
GRID_LAYOUT = "cells"


def device_grid(torch, prim, gp, device):
    """A grid on the device in the bench's layout: the plane-layout array as uploaded, or
    repacked once into the cell layout by the library (like the upload, outside any timing).
    Returns (tensor, grid parameters)."""
    from paper_2203_15963_gb300 import images
    p = prim if torch.is_tensor(prim) else torch.from_numpy(prim)
    p = p.to(device)
    if GRID_LAYOUT == "cells":
        return images.pack_grid(p, gp)
    return p, gp


def build_workload(torch, precision_code, device, case="full"):
    from paper_2203_15963_gb300 import synth as S
    gp = S.grid_params_for(*GRID)
    spins, incs = (SPINS, INCS) if case == "full" else ((0.94,), (60.0,))
    prims_host, prims, planes = {}, {}, {}
    for spin in spins:
        prims_host[spin] = S.make_torus(gp, spin, S.BASE_SEED + 1)
        planes[spin] = torch.from_numpy(prims_host[spin]).to(device)
        prims[spin], gpd = device_grid(torch, planes[spin], gp, device)
    cams, mets, gps, ps, pls, freqs = [], [], [], [], [], []
    for spin in spins:
        for inc in incs:
            cams.append(S.Camera(theta=math.radians(inc), n=N_PIX))
            mets.append(S.Metric(spin=spin, precision=precision_code))
            gps.append(gpd)
            ps.append(prims[spin])
            pls.append(planes[spin])
            freqs.append(FREQ)
    # gps/prims: the device grids as traced; gp/prims_planes: the same grids in the plane
    # layout (host arrays for the oracle and the host-buffer path, device copies for comparison)
    return dict(gp=gp, cams=cams, mets=mets, gps=gps, prims=ps, freqs=freqs,
                prims_host=prims_host, prims_planes=pls)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [ln.split(",") for ln in open(self.path).read().splitlines() if ln.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(wl, n_per_image, seed=99, single_thread=False):
    """The oracle, as it stands, on a bounded sample of the same workload (all host cores)."""
    import numpy as np
    import oracle as O
    O.build()
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    rays = 0
    for cam, met, spin in zip(wl["cams"], wl["mets"], [m.spin for m in wl["mets"]]):
        gp = wl["gp"]
        pix = np.sort(rng.choice(cam.n * cam.n, n_per_image, replace=False)).astype(np.int32)
        O.trace(cam, met, gp, wl["prims_host"][spin], FREQ, pix=pix, nthreads=0)
        rays += n_per_image
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    out = {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
           "sample": f"{n_per_image} seeded pixels from each of the 9 images ({rays} rays), "
                     f"{dt:.1f} s wall on {cores} threads", "cpu": _cpu_model()}
    if single_thread:
        # one thread on a smaller sample of the same images
        t0 = time.perf_counter()
        n1 = 0
        for cam, met in zip(wl["cams"], wl["mets"]):
            gp = wl["gp"]
            pix = np.sort(rng.choice(cam.n * cam.n, 16, replace=False)).astype(np.int32)
            O.trace(cam, met, gp, wl["prims_host"][met.spin], FREQ, pix=pix, nthreads=1)
            n1 += 16
        out["single_thread"] = {"value": n1 / (time.perf_counter() - t0), "rays": n1}
    return out


def _cpu_model():
    """the host CPU's model name, as the system reports it"""
    try:
        import subprocess
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    wl = build_workload_host()
    n_per_image = 128
    for _ in range(args.warmup):
        cpu_baseline(wl, n_per_image, seed=1)
    vals, t_total = [], 0.0
    for k in range(args.steps):
        r = cpu_baseline(wl, n_per_image, seed=100 + k)
        vals.append(r["value"])
    value = statistics.median(vals)
    ms = 9 * n_per_image / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "torus256_cam256", "images": 9, "camera": N_PIX,
                       "grid": list(GRID), "spins": list(SPINS), "inclinations_deg": list(INCS),
                       "freq_ghz": FREQ / 1e9, "sample_per_step": f"{n_per_image} pixels x 9 images"},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": os.cpu_count() or 1,
                             "kind": "oracle",
                             "sample": f"{n_per_image} seeded pixels from each of the 9 images per step"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def build_workload_host():
    from paper_2203_15963_gb300 import synth as S
    gp = S.grid_params_for(*GRID)
    prims_host = {spin: S.make_torus(gp, spin, S.BASE_SEED + 1) for spin in SPINS}
    cams, mets, gps = [], [], []
    for spin in SPINS:
        for inc in INCS:
            cams.append(S.Camera(theta=math.radians(inc), n=N_PIX))
            mets.append(S.Metric(spin=spin))
            gps.append(gp)
    return dict(gp=gp, cams=cams, mets=mets, gps=gps, prims_host=prims_host)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)
    from paper_2203_15963_gb300 import images, native
    native.build()
    native.load()
    global GRID_LAYOUT
    GRID_LAYOUT = args.grid_layout
    prec = {"mixed": native.BL_PREC_MIXED, "fp64": native.BL_PREC_FP64,
            "fast": native.BL_PREC_FAST}[args.precision]
    wl = build_workload(torch, prec, device, args.case)
    cams, mets = wl["cams"], wl["mets"]
    ws = torch.empty(native.blacklight_workspace_size(cams, mets), dtype=torch.uint8,
                     device=device)
    dt = torch.float64 if prec == native.BL_PREC_FP64 else torch.float32
    outs = [images.alloc_outputs(c.n, dt, device=device, samples=True) for c in cams]
    rays_per_step = sum(c.n * c.n for c in cams)

    coef_mlp = None
    if args.coef == "mlp":
        # the learned coefficient model in the transfer (trained here, outside the timing)
        from paper_2203_15963_gb300 import coefmodel
        coef_mlp, _ = coefmodel.train(device=device)

    def step():
        return native.blacklight_trace_batch(cams, mets, wl["gps"], wl["prims"], wl["freqs"],
                                             outs, workspace=ws, flags=native.BL_TIMING,
                                             coef_mlp=coef_mlp)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(device.index)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    native.blacklight_launch_count(reset=True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    geo_ms, tr_ms, rcs = 0.0, 0.0, []
    e0.record(stream)
    for _ in range(args.steps):
        rcs.append(step())
        g, t = native.blacklight_last_kernel_ms()
        geo_ms += g
        tr_ms += t
    e1.record(stream)
    torch.cuda.synchronize()
    launches = native.blacklight_launch_count()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed = reduce_elapsed(torch, e0.elapsed_time(e1) / 1e3, world, device)
    value = weak_scaling_value(world, rays_per_step, args.steps, elapsed)

    # algorithmic work of one launch pair (identical every step)
    attempts = sum(int(o["steps"].long().sum()) for o in outs)
    samples = sum(int(o["samples"].long().sum()) for o in outs)
    geo_avg = geo_ms / args.steps / 1e3
    tr_avg = tr_ms / args.steps / 1e3
    flop_geo = attempts * FLOP64_PER_ATTEMPT
    flop_tr = samples * FLOP32_PER_SAMPLE
    if geo_avg >= tr_avg and prec != native.BL_PREC_FAST:
        roof = {"kernel": "geodesic_kernel (FP64)", "bound": "alu",
                "achieved": flop_geo / geo_avg / 1e12, "peak": PEAK_FP64_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "nominal FP64 rate (profiling recipe)"}
    elif geo_avg >= tr_avg:
        # double-float: algorithmic FP64 flops against the emulated rate the FP32 pipe allows
        roof = {"kernel": "geodesic_kernel (double-float on FP32)", "bound": "alu",
                "achieved": flop_geo / geo_avg / 1e12, "peak": PEAK_DF64_TFLOPS,
                "unit": "TFLOP/s",
                "peak_source": f"FP32 issue rate (152 SMs x 128 lanes x 2.07 GHz) / "
                               f"{DF64_INSTR_PER_FLOP} FP32 instructions per emulated FP64 flop"}
    else:
        peak = PEAK_FP32_TFLOPS if prec != native.BL_PREC_FP64 else PEAK_FP64_TFLOPS
        roof = {"kernel": "transfer_kernel", "bound": "alu",
                "achieved": flop_tr / tr_avg / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "nominal rate (profiling recipe unit counts x 2.07 GHz)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes (read + written) of the dominant kernel per launch: the per-unit figure from
    # one ncu capture of the same kernel on the one-image 256^2 case, scaled by the units of
    # this launch (attempts for the geodesic kernel, samples for the transfer kernel)
    if (roof["kernel"].startswith("geodesic_kernel (double-float")
            and GEO_DF64_DRAM_BYTES_PER_ATTEMPT is not None):
        roof["traffic"] = GEO_DF64_DRAM_BYTES_PER_ATTEMPT * attempts
        roof["traffic_note"] = "ncu capture of the 256^2 one-image case, scaled by DP attempts"
    else:
        roof["traffic"] = None
    status_bad = sum(int(((o["status"] != 1) & (o["status"] != 2)).sum()) for o in outs)
    # the secondary measurements below allocate their own workspaces
    del ws
    torch.cuda.empty_cache()

    other = None
    if not args.no_other_forms:
        other = {}
        for name, code in (("mixed", native.BL_PREC_MIXED), ("fp64", native.BL_PREC_FP64),
                           ("fast", native.BL_PREC_FAST)):
            if code == prec:
                continue
            other[name] = time_form(torch, native, images, wl, code, device, steps=3, warmup=2)
    layout_cmp = None
    if not args.no_other_forms and GRID_LAYOUT == "cells":
        # the same step on the grids in the plane layout (the layout as generated)
        wl_planes = dict(wl, gps=[wl["gp"]] * len(cams), prims=wl["prims_planes"])
        layout_cmp = time_form(torch, native, images, wl_planes, prec, device, steps=3, warmup=2)
    hires = hires_img = None
    if not args.no_hires and args.case == "full":
        hires, hires_img = measure_hires(torch, native, images, prec, device,
                                         keep_image=prec == native.BL_PREC_FAST)
    variants = None
    if not args.no_variants:
        variants = measure_variants(torch, native, images, wl, prec, device)
    plan = None
    if not args.no_plan:
        plan = measure_plan(torch, native, images, wl, prec, device)
    model = None
    if (not args.no_mlp or not args.no_slow) and args.case == "full":
        from paper_2203_15963_gb300 import coefmodel
        t0 = time.perf_counter()
        params, hist = coefmodel.train(device=device)
        torch.cuda.synchronize()
        model = (params, time.perf_counter() - t0, float(hist[-500:].mean()))
    mlp = None
    if not args.no_mlp and args.case == "full":
        mlp = measure_mlp(torch, native, images, device, hires_img, *model)
    hires_img = None
    slow = None
    if not args.no_slow and args.case == "full":
        slow = measure_slow(torch, native, images, device, model[0] if model else None)
    model = None
    adaptive = None
    if not args.no_adaptive and args.case == "full":
        adaptive = measure_adaptive(torch, native, prec, device)
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(torch, native, wl, prec, max(1, min(args.steps, 3)))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, 1024, single_thread=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {native.BL_PREC_MIXED: "f64+f32", native.BL_PREC_FP64: "f64",
                          native.BL_PREC_FAST: "df64+f32"}[prec],
                "data": "synthetic",
                "config": {"workload": "torus256_cam256" if args.case == "full"
                           else "torus256_cam256 (one image: a=0.94, i=60 deg)",
                           "images": len(cams), "camera": N_PIX,
                           "grid": list(GRID), "spins": list(SPINS),
                           "inclinations_deg": list(INCS), "freq_ghz": FREQ / 1e9,
                           "precision": args.precision, "coefficients": args.coef,
                           "grid_layout": GRID_LAYOUT,
                           "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (3 x 134 MB grids + sample records); no flush"},
                "kernel_ms": {"geodesic": geo_avg * 1e3, "transfer": tr_avg * 1e3},
                "work": {"dp_attempts": attempts, "samples": samples,
                         "rays_not_terminated_normally": status_bad},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "other_forms": other,
                "plane_layout": layout_cmp,
                "variants": variants, "plan": plan, "hires": hires, "mlp": mlp,
                "slow_light": slow,
                "adaptive": adaptive,
                "gpu_launches": int(launches), "clocks": clk, "return_codes": sorted(set(rcs))}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def time_form(torch, native, images, wl, code, device, steps, warmup):
    """Short CUDA-event timing of the same workload in another precision form."""
    import copy
    mets = [copy.replace(m, precision=code) if hasattr(copy, "replace") else
            type(m)(**{**m.__dict__, "precision": code}) for m in wl["mets"]]
    cams = wl["cams"]
    ws = torch.empty(native.blacklight_workspace_size(cams, mets), dtype=torch.uint8,
                     device=device)
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    outs = [images.alloc_outputs(c.n, dt, device=device) for c in cams]
    for _ in range(warmup):
        native.blacklight_trace_batch(cams, mets, wl["gps"], wl["prims"], wl["freqs"], outs,
                                      workspace=ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    geo = tr = 0.0
    e0.record()
    for _ in range(steps):
        native.blacklight_trace_batch(cams, mets, wl["gps"], wl["prims"], wl["freqs"], outs,
                                      workspace=ws, flags=native.BL_TIMING)
        g, t = native.blacklight_last_kernel_ms()
        geo += g
        tr += t
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del ws
    rays = sum(c.n * c.n for c in cams)
    return {"value": rays / ms * 1e3, "ms_per_step": ms, "steps": steps,
            "kernel_ms": {"geodesic": geo / steps, "transfer": tr / steps}}


def measure_hires(torch, native, images, code, device, steps=3, warmup=2, coef_mlp=None,
                  keep_image=False):
    """The metric's 1024^2 point: one 1024x1024 image (a = 0.94, i = 17 deg, 230 GHz) on the
    512x256x256 torus (1 GiB of float32), timed like the main workload. coef_mlp selects the
    learned coefficient model. Returns (line, Stokes image or None)."""
    from paper_2203_15963_gb300 import synth as S
    cam, met, gp, prim = S.workload_inputs("torus512_cam1024", 0.94, 17.0)
    met = S.Metric(**{**met.__dict__, "precision": code})
    p, gp = device_grid(torch, prim, gp, device)
    del prim
    ws = torch.empty(native.blacklight_workspace_size([cam], [met]), dtype=torch.uint8,
                     device=device)
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    out = images.alloc_outputs(cam.n, dt, device=device)
    for _ in range(warmup):
        native.blacklight_trace_batch([cam], [met], [gp], [p], [FREQ], [out], workspace=ws,
                                      coef_mlp=coef_mlp)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    geo = tr = 0.0
    e0.record()
    for _ in range(steps):
        native.blacklight_trace_batch([cam], [met], [gp], [p], [FREQ], [out], workspace=ws,
                                      flags=native.BL_TIMING, coef_mlp=coef_mlp)
        g, t = native.blacklight_last_kernel_ms()
        geo += g
        tr += t
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    bad = int(((out["status"] != 1) & (out["status"] != 2)).sum())
    del ws, p
    torch.cuda.empty_cache()
    line = {"workload": "torus512_cam1024", "value": cam.n * cam.n / ms * 1e3, "unit": "rays/s",
            "ms_per_step": ms, "steps": steps,
            "kernel_ms": {"geodesic": geo / steps, "transfer": tr / steps},
            "rays_not_terminated_normally": bad}
    return line, (out["stokes"] if keep_image else None)


def rel_l2(torch, got, want):
    """per-Stokes ||got - want|| / ||I_want|| of two [4][n][n] images"""
    g, w = got.double(), want.double()
    nI = torch.linalg.vector_norm(w[0])
    return [float(torch.linalg.vector_norm(g[s] - w[s]) / nI) for s in range(4)]


def measure_slow(torch, native, images, device, coef_mlp, steps=3):
    """Slow light: 8 snapshots (10 M apart) of the 256x128x128 rotating torus, one 512^2 image
    (a = 0.94, i = 60 deg, 230 GHz), traced through a plan (CUDA-graph replay): fast form with
    the exact fits, and mixed form with the learned coefficients; the fast-light image of the
    middle snapshot alone for comparison."""
    import dataclasses
    from paper_2203_15963_gb300 import synth as S
    cam, met, gp, prim = S.workload_inputs("torus256_slow8_cam512", 0.94, 60.0)
    p, gp = device_grid(torch, prim, gp, device)
    mid = p[4].contiguous()       # the middle snapshot alone, in the same layout
    del prim

    def run(gpx, px, code, mlp):
        m = S.Metric(**{**met.__dict__, "precision": code})
        outs = [images.alloc_outputs(cam.n, torch.float32, device=device)]
        plan = native.Plan([cam], [m], [gpx], [px], [FREQ], outs, coef_mlp=mlp)
        plan.run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.run()
        e1.record()
        torch.cuda.synchronize()
        rc = plan.check()
        plan.close()
        ms = e0.elapsed_time(e1) / steps
        return {"value": cam.n * cam.n / ms * 1e3, "ms_per_step": ms, "return_code": rc}, outs[0]["stokes"]

    slow, img = run(gp, p, native.BL_PREC_FAST, None)
    out = {"workload": "torus256_slow8_cam512", "unit": "rays/s", "steps": steps,
           "slow_fast_exact": slow}
    if coef_mlp is not None:
        slow_mlp, img_mlp = run(gp, p, native.BL_PREC_MIXED, coef_mlp)
        slow_mlp["image_rel_l2_vs_exact_fits"] = rel_l2(torch, img_mlp, img)
        out["slow_mixed_learned"] = slow_mlp
    fast, img_fast = run(dataclasses.replace(gp, n_snapshots=1), mid, native.BL_PREC_FAST, None)
    fast["image_rel_l2_slow_vs_this"] = rel_l2(torch, img, img_fast)
    out["fast_light_middle_snapshot"] = fast
    del p, mid, img
    torch.cuda.empty_cache()
    return out


def measure_mlp(torch, native, images, device, fast_image, params, train_s, final_loss):
    """Learned coefficients at the 1024^2 point: the model trained on the GPU (default recipe),
    then the image traced with the fused tensor-core transfer (double-float geodesics, FP32
    transfer), next to the plain FP64 form of the same image: speedup and image error
    against the FP64 image, and the exact-fit fast form's error for comparison."""
    from paper_2203_15963_gb300 import coefmodel
    line, img = measure_hires(torch, native, images, native.BL_PREC_FAST, device, steps=3,
                              warmup=2, coef_mlp=params, keep_image=True)
    fp64, img64 = measure_hires(torch, native, images, native.BL_PREC_FP64, device, steps=1,
                                warmup=1, keep_image=True)
    line.update({
        "form": "double-float geodesics, FP32 transfer, learned coefficients (BF16 tensor cores)",
        "train": {"seconds": train_s, "samples": coefmodel.N_SAMPLES, "batch": coefmodel.BATCH,
                  "steps": coefmodel.STEPS, "final_mse_normalised": final_loss},
        "fp64_form": {"value": fp64["value"], "kernel_ms": fp64["kernel_ms"]},
        "speedup_over_fp64_form": line["value"] / fp64["value"],
        "image_rel_l2_vs_fp64_form": rel_l2(torch, img, img64),
        "exact_fast_rel_l2_vs_fp64_form": (rel_l2(torch, fast_image, img64)
                                           if fast_image is not None else None)})
    del img, img64
    torch.cuda.empty_cache()
    return line


def measure_variants(torch, native, images, wl, code, device, steps=2):
    """The main workload (9 x 256^2) in the method's other modes: unpolarized transfer
    (Eq. unpolarized), polarized with the 26 auxiliary images, and the fixed-rule RK4 and RK2
    integrators (f_step = 0.02, FP64 geodesics). Device time per step, CUDA events."""
    import dataclasses
    cams = wl["cams"]
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    rays = sum(c.n * c.n for c in cams)

    def run(mets, flags=0, aux=False):
        outs = [images.alloc_outputs(c.n, dt, device=device, aux=aux) for c in cams]
        native.blacklight_trace_batch(cams, mets, wl["gps"], wl["prims"], wl["freqs"], outs,
                                      flags=flags)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            rc = native.blacklight_trace_batch(cams, mets, wl["gps"], wl["prims"], wl["freqs"],
                                               outs, flags=flags)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        del outs
        torch.cuda.empty_cache()
        return {"value": rays / ms * 1e3, "ms_per_step": ms, "return_code": rc}

    out = {"unit": "rays/s", "steps": steps,
           "unpolarized": run(wl["mets"], flags=native.BL_UNPOLARIZED),
           "polarized_with_aux": run(wl["mets"], aux=True)}
    for name, integ in (("rk4", native.BL_INT_RK4), ("rk2", native.BL_INT_RK2)):
        mets = [dataclasses.replace(m, integrator=integ, f_step=0.02) for m in wl["mets"]]
        out[name + "_f0.02"] = run(mets)
    return out


def measure_plan(torch, native, images, wl, code, device, steps=5):
    """The main workload as an autotuned plan (CUDA-graph replay), device-timed like the
    headline, and the host cost of small batches (16 images of 32^2 on the 64x32x32 torus)
    through direct calls against graph replays (wall clock per batch, synchronised)."""
    from paper_2203_15963_gb300 import synth as S
    cams, mets = wl["cams"], wl["mets"]
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    outs = [images.alloc_outputs(c.n, dt, device=device) for c in cams]
    t0 = time.perf_counter()
    plan = native.Plan(cams, mets, wl["gps"], wl["prims"], wl["freqs"], outs, autotune=True)
    tune_s = time.perf_counter() - t0
    cfg = plan.config()
    for _ in range(2):
        plan.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.run()
    e1.record()
    torch.cuda.synchronize()
    rc = plan.check()
    ms = e0.elapsed_time(e1) / steps
    rays = sum(c.n * c.n for c in cams)
    plan.close()
    del outs
    # small batches: host overhead of direct calls against replays
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 17.0)
    met = S.Metric(**{**met.__dict__, "precision": code})
    p, gp = device_grid(torch, prim, gp, device)
    k = 16
    cs, ms_, gs, ps, fs = [cam] * k, [met] * k, [gp] * k, [p] * k, [FREQ] * k
    so = [images.alloc_outputs(cam.n, dt, device=device) for _ in range(k)]
    ws = torch.empty(native.blacklight_workspace_size(cs, ms_), dtype=torch.uint8, device=device)
    small = native.Plan(cs, ms_, gs, ps, fs, so)

    def wall(fn, n=20):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / n * 1e3

    direct_ms = wall(lambda: native.blacklight_trace_batch(cs, ms_, gs, ps, fs, so, workspace=ws,
                                                           flags=native.BL_ASYNC))
    replay_ms = wall(small.run)
    small.close()
    del ws, so, p
    torch.cuda.empty_cache()
    return {"value": rays / ms * 1e3, "unit": "rays/s", "ms_per_step": ms, "steps": steps,
            "return_code": rc, "autotune_seconds": tune_s, "config": cfg,
            "small_batch": {"workload": "16 x 32^2 on the 64x32x32 torus",
                            "direct_ms": direct_ms, "graph_replay_ms": replay_ms}}


def measure_adaptive(torch, native, code, device, steps=2, warmup=1):
    """Batched adaptive refinement: 16 images (spins 0, 0.5, 0.94, 0.99 x 86, 230, 345, 690 GHz)
    on the 256x128x128 torus, 128^2 root pixels in 8x8 blocks, up to 3 levels, refining blocks
    where the relative Stokes-I gradient exceeds 0.1 on at least 5 of 64 pixels."""
    from paper_2203_15963_gb300 import synth as S
    gp = S.grid_params_for(*GRID)
    spins, freqs = (0.0, 0.5, 0.94, 0.99), (86e9, 230e9, 345e9, 690e9)
    prims = {}
    for a in spins:
        prims[a], gpd = device_grid(torch, S.make_torus(gp, a, S.BASE_SEED + 2), gp, device)
    gp = gpd
    cams, mets, gps, ps, fs, outs = [], [], [], [], [], []
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    for a in spins:
        for f in freqs:
            cams.append(S.Camera(theta=math.radians(17.0), n=128))
            mets.append(S.Metric(spin=a, precision=code))
            gps.append(gp)
            ps.append(prims[a])
            fs.append(f)
            outs.append({"stokes": torch.zeros((4, 1024, 1024), dtype=dt, device=device)})
    ad = native.adapt_struct(8, 3, native.BL_CRIT_REL_GRAD, 0.1, 5)
    for _ in range(warmup):
        native.blacklight_trace_adaptive(cams, mets, gps, ps, fs, ad, outs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        rc, lr = native.blacklight_trace_adaptive(cams, mets, gps, ps, fs, ad, outs)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / steps
    rays = int(lr.sum())
    # the same trace as an adaptive plan: every level in one CUDA graph, device-timed
    plan = native.AdaptivePlan(cams, mets, gps, ps, fs, ad, outs)
    plan.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.run()
    e1.record()
    torch.cuda.synchronize()
    plan_ms = e0.elapsed_time(e1) / steps
    plan_rc = plan.check()
    plan_rays = int(plan.level_rays().sum())
    plan.close()
    del prims, ps, outs
    torch.cuda.empty_cache()
    return {"workload": "torus256 adaptive: 16 images, 128^2 root, 8x8 blocks, 3 levels",
            "value": rays / sec, "unit": "rays/s", "ms_per_step": sec * 1e3, "steps": steps,
            "rays_per_step": rays, "rays_per_level": lr.sum(axis=0).tolist(),
            "timing": "host wall clock of blacklight_trace_adaptive (levels run on the device "
                      "without host round trips; one synchronisation at the end)",
            "graph_plan": {"value": plan_rays / plan_ms * 1e3, "ms_per_step": plan_ms,
                           "return_code": plan_rc, "timing": "CUDA events around graph replays"}}


def measure_e2e(torch, native, wl, prec, steps):
    """Same workload through the C ABI's host-buffer entry point: per step, one
    blacklight_trace_host_batch call copies the three grids (one per spin, shared by that
    spin's images) from pinned host memory, traces the 9 images in one batched launch and
    copies the 9 Stokes images back, all inside the timing (the library repacks each grid
    into the cell layout on the device as part of the call)."""
    host_prims = {s: torch.from_numpy(p).pin_memory() for s, p in wl["prims_host"].items()}
    dt = torch.float64 if prec == native.BL_PREC_FP64 else torch.float32
    outs = [{"stokes": torch.empty((4, c.n, c.n), dtype=dt).pin_memory()} for c in wl["cams"]]
    h2d = sum(p.numel() * 4 for p in host_prims.values())
    d2h = sum(o["stokes"].numel() * o["stokes"].element_size() for o in outs)
    prims = [host_prims[m.spin] for m in wl["mets"]]
    # keep the library's stream-ordered scratch reserved between calls (a host application
    # tracing repeatedly would do the same); restored to the CUDA default afterwards
    native.blacklight_set_memory_retention(2 ** 64 - 1)

    def one():
        native.blacklight_trace_host_batch(wl["cams"], wl["mets"], [wl["gp"]] * len(prims),
                                           prims, wl["freqs"], outs)

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt_s = (time.perf_counter() - t0) / steps
    native.blacklight_set_memory_retention(0)
    rays = sum(c.n * c.n for c in wl["cams"])
    return {"value": rays / dt_s, "unit": "rays/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps,
            "path": "blacklight_trace_host_batch (pinned host grids in, Stokes out; "
                    "scratch retained in the memory pool between calls)"}


if __name__ == "__main__":
    main()
