#!/usr/bin/env python
"""Benchmark of the Blacklight hot path on GB300: rays/s of geodesic + polarized transfer.

Workload (one step): 9 images -- spins {0, 0.5, 0.94} x inclinations {17, 60, 90} deg -- of
256x256 pixels each, camera at r = 1000 M with a +-20 M field of view, 230 GHz, on the seeded
synthetic torus sampled on a 256x128x128 spherical Kerr-Schild grid (one grid per spin), traced
in one batched persistent launch pair. Inputs stay resident in HBM; the three grids (3 x 134 MB)
plus the per-sample records exceed the 129 MB L2, so no explicit flush is needed between steps.

The headline is the FP64 form (geodesics, sampling, plasma, coefficients and transfer all in
IEEE double, the arithmetic of the paper's C++ code); the mixed (FP64 geodesics, FP32
transfer) and fast (double-float geodesics, FP32 transfer) forms are secondary lines, each
with its image error against the CPU oracle on a seeded pixel sample.

Rooflines: achieved = algorithmic flops per launch / the kernel's CUDA-event time, against
the device's own peak measured by blacklight_measure_peaks (FMA-chain probes for FP64, FP32
and the double-float arithmetic), with the SM clock sampled while the probes run.
  - geodesic kernel: FLOP64_PER_ATTEMPT per Dormand-Prince attempt (hand count below), and in
    the FP64 form FLOP64_EMIT_PER_RECORD per sample record for its FP64 sample emission;
  - transfer kernel: FLOP_PER_SAMPLE per sample, the method's arithmetic per sample as the
    FP32 transfer kernel executes it with the stencil field test on (ncu thread-level FFMA x 2
    + FADD + FMUL per sample; its special functions are single hardware instructions, counted
    apart in SFU_PER_SAMPLE). The FP64 passes run the same source with the same test, so the
    same count is their algorithmic work; their FP64 special-function sequences are overhead
    on top of it.
DRAM traffic per launch comes from one ncu capture per kernel (per-unit figure x the units of
the launch) and is reported only while the kernel sources still hash to those captured.

Rank 0 prints one JSON line. Under torchrun each rank traces its own share of the images
(weak scaling, see `rank_images`); there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
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
# FP64 flops per Dormand-Prince attempt, counted by hand from the method as implemented: 6
# right-hand sides of 114 flops (81 products, 30 sums, 2 reciprocal square roots, 1
# reciprocal, with d_c(l.k) formed directly), 6 stage combinations (384), the embedded error
# estimate (96) and its norm and the step control (50).
FLOP64_PER_ATTEMPT = 1214
# FP64 flops per sample record of the sample emission inside the geodesic kernel (Sec. 2.2's
# sample points), a lower bound counted from the method as implemented, FP64 form only (the
# other forms emit their records in FP32): an accepted step that is not subdivided costs 136
# (Shampine midpoint 91 over the 7 varying components, geometry at the midpoint 35, L and
# k^t 8, ds 2) for its one record; a step split into n sub-samples costs 242 + 108 n (the
# midpoint and geometry, the quartic's coefficients 154, then a sample point 56, a node 48 and
# 4 for its parameters and length a record, the first node being the step's start), i.e. at
# least 108 a record.
FLOP64_EMIT_PER_RECORD = 108
# Arithmetic per transfer sample of the method (see the module docstring): FP32 flops and
# special-function instructions of transfer_kernel<float, float, 0> per sample with the
# stencil field test on (a sample whose lookup stencil carries no magnetic field stops after
# the lookup), from the ncu capture of the one-image 256^2 case on plane-layout grids (a =
# 0.94, i = 60 deg; 18,372,183 samples): 2 x 4.397e9 FFMA + 2.661e9 FMUL + 0.703e9 FADD
# thread instructions, 2.43e8 MUFU. (Without the test, as the cell-layout FP32 transfer runs
# for its record-count queue, the kernel executes 848 flops a sample: the difference is work
# the method does not need.)
FLOP_PER_SAMPLE = 662
SFU_PER_SAMPLE = 13.2
# The CUDA kernel headers (their code hash is printed with the results), and the ones the
# kernels of the table below are built from: the geodesic and exact-fit transfer kernels
# instantiate nothing of the learned model's headers (bl_mlp.cuh, bl_tc.cuh), so a change
# there leaves their captured figures valid.
KERNEL_HEADERS = ("bl_kernels.cuh", "bl_math.cuh", "bl_df64.cuh", "bl_internal.cuh",
                  "bl_mlp.cuh", "bl_tc.cuh")
TRAFFIC_HEADERS = ("bl_kernels.cuh", "bl_math.cuh", "bl_df64.cuh", "bl_internal.cuh")
# dram__bytes_read.sum + dram__bytes_write.sum per unit of work from one ncu capture of the
# one-image 256^2 case, with the kernel-source hash of that capture; scaled by the units of a
# launch of the benchmark step (the kernels' traffic grows with the units they process).
# fp64_instr: thread-level DFMA + DMUL + DADD instructions per unit from the same capture,
# which gives the FP64 pipe's issue rate beside the algorithmic roofline.
DRAM_PER_UNIT = {
    # FP64 form, 7,845,751 attempts: 0.677 GB read + 5.398 GB written (the FP64 records and the
    # stage derivatives, held in local memory at 16 CTAs an SM)
    "geodesic_fp64": {"src": "c20dc1578110e077", "bytes": 774.3, "unit": "attempt",
                      "fp64_instr": 1091.2},
    # FP64 form, 18,372,204 samples, the transfer's launches: fp64_samples_kernel 4.190 + 3.815
    # GB (records, the stencils' field values, grid gathers, 193 B of results a plasma sample,
    # spills) and transport_fp64_kernel 1.501 + 2.439 GB (records, those results, spills)
    "transfer_fp64": {"src": "c20dc1578110e077", "bytes": 650.2, "unit": "sample",
                      "fp64_instr": 405.4},
    # fast form, 7,845,744 attempts: 0.026 GB read + 1.135 GB written
    "geodesic_df64": {"src": "c20dc1578110e077", "bytes": 147.9, "unit": "attempt"},
    # fast form on cell-layout grids (record-count queue, no field test), 18,372,183 samples:
    # 1.434 GB read + 0.006 GB written
    "transfer_fp32": {"src": "c20dc1578110e077", "bytes": 78.4, "unit": "sample"},
}


def source_code_text(text: str) -> str:
    """C++/CUDA source without its comments and blank lines (what the compiler sees of it)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_source_hash(headers=KERNEL_HEADERS) -> str:
    """sha256 (16 hex digits) of the code of CUDA kernel headers (by default all of them, the
    sources of every kernel the benchmark times); comments do not count: a comment edit leaves
    the kernels and their captured counters as they were."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2203_15963_gb300", "csrc")
    for f in headers:
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            h.update(source_code_text(fh.read()).encode("utf-8"))
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="blacklight", choices=["blacklight", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["mixed", "fp64", "fast"],
                    help="fp64: FP64 throughout (default, the headline); mixed: FP64 geodesics + "
                         "FP32 transfer; fast: double-float geodesics + FP32 transfer")
    ap.add_argument("--no-other-forms", action="store_true",
                    help="skip the short timing of the two other precision forms")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: one 256^2 image (a=0.94, i=60 deg) of the same workload, for "
                         "profiler captures")
    ap.add_argument("--grid-layout", default="cells", choices=["cells", "planes"],
                    help="memory order of the device grids: cells (repacked once by "
                         "blacklight_grid_pack) or planes (as generated)")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the FP64/FP32/double-float peak probes (rooflines then unreported)")
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
    ap.add_argument("--oracle-pixels", type=int, default=4096,
                    help="seeded pixels per image the CPU oracle traces for the baseline and the "
                         "image-error comparisons")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_elapsed(torch, elapsed, world, device):
    """Slowest rank's timed-region length (ranks trace disjoint shares, no exchange)."""
    if world <= 1:
        return elapsed
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, rays_per_rank_step, steps, elapsed_max):
    """Whole-job rays/s: every rank's rays over the slowest rank's time."""
    return world * rays_per_rank_step * steps / elapsed_max


def image_spec(k, world):
    """Image k of the whole job's batch of 9 x world images: (spin, inclination in degrees,
    camera azimuth in radians). Images 9 w .. 9 w + 8 repeat the 9 spin x inclination pairs
    seen from the azimuth 2 pi w / world, so every rank's share has the same structure and
    cost while no two ranks trace the same image (the torus's seeded noise breaks the
    axisymmetry)."""
    w, j = divmod(k, len(SPINS) * len(INCS))
    return SPINS[j // len(INCS)], INCS[j % len(INCS)], 2.0 * math.pi * w / max(world, 1)


def rank_images(rank, world, per_rank=len(SPINS) * len(INCS)):
    """Indices of the images rank `rank` traces: a contiguous block of `per_rank` images, so
    the ranks' shares are disjoint and together cover the job's per_rank x world images."""
    return list(range(rank * per_rank, (rank + 1) * per_rank))


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


def workload_config(args, world):
    """The workload description both arms print (identical keys and values)."""
    small = args.case == "small"
    return {"workload": "torus256_cam256" if not small
            else "torus256_cam256 (one image: a=0.94, i=60 deg)",
            "images": 1 if small else len(SPINS) * len(INCS) * world,
            "images_per_rank": 1 if small else len(SPINS) * len(INCS),
            "camera": N_PIX, "grid": list(GRID), "spins": list(SPINS),
            "inclinations_deg": list(INCS), "freq_ghz": FREQ / 1e9,
            "precision": args.precision, "coefficients": args.coef,
            "grid_layout": args.grid_layout,
            "parallelism": f"{world} rank(s), disjoint image shares, no collective",
            "l2": "inputs larger than L2 (3 x 134 MB grids + sample records); no flush"}


def build_workload(torch, precision_code, device, case="full", rank=0, world=1):
    from paper_2203_15963_gb300 import synth as S
    gp = S.grid_params_for(*GRID)
    if case == "full":
        specs = [image_spec(k, world) for k in rank_images(rank, world)]
    else:
        specs = [(0.94, 60.0, 0.0)]
    prims_host, prims, planes = {}, {}, {}
    for spin in sorted({sp[0] for sp in specs}):
        prims_host[spin] = S.make_torus(gp, spin, S.BASE_SEED + 1)
        planes[spin] = torch.from_numpy(prims_host[spin]).to(device)
        prims[spin], gpd = device_grid(torch, planes[spin], gp, device)
    cams, mets, gps, ps, pls, freqs = [], [], [], [], [], []
    for spin, inc, phi in specs:
        cams.append(S.Camera(theta=math.radians(inc), phi=phi, n=N_PIX))
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


def measure_peaks(native, device):
    """The device's measured FP64, FP32 and double-float multiply-add peaks, with the SM
    clock sampled while the probes run."""
    clk = ClockSampler(device.index)
    clk.start()
    time.sleep(0.25)
    pk = native.blacklight_measure_peaks(reps=20)
    time.sleep(0.25)
    pk["clocks"] = clk.stop()
    pk["how"] = ("blacklight_measure_peaks: FMA-chain kernels (8 independent chains a thread, "
                 "full occupancy on every SM), best of 20 launches, CUDA events")
    return pk


def roofline(kernel, flops_per_unit, units, unit_name, seconds, peak, traffic_key=None,
             note=None):
    """One roofline entry: algorithmic flops of a launch over its measured time against the
    measured peak `peak` = (TFLOP/s, source); traffic from DRAM_PER_UNIT when the kernel
    sources are the ones captured."""
    r = {"kernel": kernel, "bound": "alu", "unit": "TFLOP/s",
         "units_per_launch": units, "work_unit": unit_name,
         "flops_per_unit": flops_per_unit, "seconds_per_launch": seconds}
    if flops_per_unit is None or peak is None or seconds <= 0:
        r.update(achieved=None, peak=None if peak is None else peak[0], frac=None,
                 peak_source=None if peak is None else peak[1])
    else:
        ach = flops_per_unit * units / seconds / 1e12
        r.update(achieved=ach, peak=peak[0], frac=ach / peak[0], peak_source=peak[1])
    r["traffic"] = None
    if traffic_key is not None:
        prof = DRAM_PER_UNIT.get(traffic_key)
        if prof is not None and prof["src"] == kernel_source_hash(TRAFFIC_HEADERS):
            r["traffic"] = prof["bytes"] * units
            r["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum per " +
                                 prof["unit"] + " from one ncu capture of the one-image 256^2 "
                                 "case, scaled by this launch's units")
            if "fp64_instr" in prof and peak is not None and seconds > 0:
                rate = prof["fp64_instr"] * units / seconds / 1e9
                r["fp64_pipe_issue"] = {
                    "ginstr_per_s": rate, "peak_ginstr_per_s": peak[0] * 1e3 / 2,
                    "frac": rate / (peak[0] * 1e3 / 2),
                    "note": "DFMA + DMUL + DADD thread instructions per unit from the ncu "
                            "capture (special-function sequences included) x units / time, "
                            "against the measured FP64 FMA rate in instructions"}
        elif prof is not None:
            r["traffic_note"] = "kernel changed since the ncu capture: traffic not reported"
    if note:
        r["note"] = note
    return r


def form_rooflines(prec_name, attempts, samples, geo_s, tr_s, peaks):
    """Rooflines of the geodesic and transfer kernels of one precision form; the dominant
    (longer) kernel first."""
    def pk(kind):
        if not peaks:
            return None
        mhz = (peaks.get("clocks") or {}).get("sm_mhz")
        return (peaks[kind + "_tflops"],
                f"measured {kind.upper()} peak ({peaks['how']}; {peaks['sm_count']} SMs"
                + (f", median SM clock {mhz:.0f} MHz during the probes)" if mhz else ")"))
    geo_kind = {"fp64": "fp64", "mixed": "fp64", "fast": "df64"}[prec_name]
    tr_kind = "fp64" if prec_name == "fp64" else "fp32"
    geo_flops, geo_note = FLOP64_PER_ATTEMPT, None
    if prec_name == "fp64" and attempts > 0:
        # the FP64 form's sample emission (FP64 records) is part of the kernel's method work
        geo_flops = FLOP64_PER_ATTEMPT + FLOP64_EMIT_PER_RECORD * samples / attempts
        geo_note = (f"algorithmic flops: {FLOP64_PER_ATTEMPT} a Dormand-Prince attempt plus at "
                    f"least {FLOP64_EMIT_PER_RECORD} a sample record of the FP64 sample emission "
                    f"({samples} records for {attempts} attempts)")
    geo = roofline({"fp64": "geodesic_kernel_fp64",
                    "mixed": "geodesic_kernel<float, double>",
                    "fast": "geodesic_kernel<float, df64>"}[prec_name],
                   geo_flops, attempts, "DP attempt", geo_s, pk(geo_kind),
                   traffic_key={"fp64": "geodesic_fp64", "fast": "geodesic_df64"}.get(prec_name),
                   note=geo_note)
    tr = roofline("transfer phase: fp64_samples_kernel + transport_fp64_kernel"
                  if prec_name == "fp64" else "transfer_kernel<float, float, 0>",
                  FLOP_PER_SAMPLE, samples, "transfer sample", tr_s, pk(tr_kind),
                  traffic_key="transfer_fp64" if prec_name == "fp64" else "transfer_fp32",
                  note=("algorithmic flops: the method's per-sample arithmetic as the FP32 "
                        f"kernel executes it ({FLOP_PER_SAMPLE} flops, plus {SFU_PER_SAMPLE} "
                        "special-function instructions not counted as flops)"))
    return (geo, tr) if geo_s >= tr_s else (tr, geo)


def _hist(v):
    """Percentiles of a per-ray count (DP attempts or sample records per ray)."""
    import numpy as np
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    if v.size == 0:
        return None
    q = np.percentile(v, [10, 50, 90, 99])
    return {"mean": float(v.mean()), "p10": float(q[0]), "p50": float(q[1]),
            "p90": float(q[2]), "p99": float(q[3]), "max": float(v.max()), "n": int(v.size)}


def cpu_baseline(wl, n_per_image, seed=99, single_thread=False):
    """The oracle, as it stands, on a bounded sample of the same workload (all host cores).
    Returns (timing line, [oracle result per image]) -- the results serve the image-error
    comparisons of the GPU forms on the same pixels."""
    import numpy as np
    import oracle as O
    O.build()
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    rays = 0
    ref = []
    for cam, met in zip(wl["cams"], wl["mets"]):
        pix = np.sort(rng.choice(cam.n * cam.n, n_per_image, replace=False)).astype(np.int32)
        ref.append(O.trace(cam, met, wl["gp"], wl["prims_host"][met.spin], FREQ, pix=pix,
                           nthreads=0))
        rays += n_per_image
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    cat = lambda k: np.concatenate([r[k] for r in ref])
    out = {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
           "sample": f"{n_per_image} seeded pixels from each of the {len(ref)} images "
                     f"({rays} rays), {dt:.1f} s wall on {cores} threads", "cpu": _cpu_model(),
           "per_core": rays / dt / cores,
           "histograms": {"dp_attempts_per_ray": _hist(cat("attempts")),
                          "accepted_steps_per_ray": _hist(cat("accepted")),
                          "samples_per_ray": _hist(cat("samples"))}}
    if single_thread:
        # one thread on a smaller sample of the same images
        t0 = time.perf_counter()
        n1 = 0
        for cam, met in zip(wl["cams"], wl["mets"]):
            pix = np.sort(rng.choice(cam.n * cam.n, 16, replace=False)).astype(np.int32)
            O.trace(cam, met, wl["gp"], wl["prims_host"][met.spin], FREQ, pix=pix, nthreads=1)
            n1 += 16
        out["single_thread"] = {"value": n1 / (time.perf_counter() - t0), "rays": n1}
    return out, ref


def oracle_image_error(outs, ref):
    """Error of GPU images against the oracle on the oracle's pixels: per Stokes the largest
    over images of ||X_gpu - X_oracle|| / ||I_oracle|| (over the sampled pixels), the
    sampled flux's largest relative difference, and ray statuses that differ."""
    import numpy as np
    worst = [0.0] * 4
    flux = 0.0
    status_diff = 0
    for o, r in zip(outs, ref):
        st = o["stokes"].double().reshape(4, -1).cpu().numpy()[:, r["pix"]].T
        want = r["stokes"]
        nI = np.linalg.norm(want[:, 0])
        for k in range(4):
            worst[k] = max(worst[k], float(np.linalg.norm(st[:, k] - want[:, k]) / nI))
        fw = float(want[:, 0].sum())
        flux = max(flux, abs(float(st[:, 0].sum()) - fw) / abs(fw) if fw else 0.0)
        if "status" in o:
            status_diff += int((o["status"].reshape(-1).cpu().numpy()[r["pix"]] != r["status"]).sum())
    return {"rel_l2_IQUV": worst, "flux_rel": flux, "status_differs": status_diff,
            "pixels": int(sum(len(r["pix"]) for r in ref))}


def _cpu_model():
    """the host CPU's model name, as the system reports it"""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def run_reference(args):
    """The oracle timed on the host cores on a bounded sample of the same workload, printed
    as a line of the same metric and config. Under torchrun only rank 0 runs it."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = build_workload_host(args, world)
    n_per_image = 128
    for _ in range(args.warmup):
        cpu_baseline(wl, n_per_image, seed=1)
    vals = []
    for k in range(args.steps):
        r, _ = cpu_baseline(wl, n_per_image, seed=100 + k)
        vals.append(r["value"])
    value = statistics.median(vals)
    n_img = len(wl["cams"])
    ms = n_img * N_PIX * N_PIX / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": os.cpu_count() or 1,
                             "kind": "oracle",
                             "sample": f"{n_per_image} seeded pixels from each of the {n_img} "
                                       f"images per step; ms_per_step extrapolates to the "
                                       f"whole step"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def build_workload_host(args, world=1):
    """The benchmark step's inputs on the host (the reference arm traces rank 0's share)."""
    from paper_2203_15963_gb300 import synth as S
    gp = S.grid_params_for(*GRID)
    specs = ([image_spec(k, world) for k in rank_images(0, world)] if args.case == "full"
             else [(0.94, 60.0, 0.0)])
    prims_host = {spin: S.make_torus(gp, spin, S.BASE_SEED + 1)
                  for spin in sorted({sp[0] for sp in specs})}
    cams, mets, gps = [], [], []
    for spin, inc, phi in specs:
        cams.append(S.Camera(theta=math.radians(inc), phi=phi, n=N_PIX))
        mets.append(S.Metric(spin=spin))
        gps.append(gp)
    return dict(gp=gp, cams=cams, mets=mets, gps=gps, prims_host=prims_host)


PREC_NAMES = ("fp64", "mixed", "fast")


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
    codes = {"mixed": native.BL_PREC_MIXED, "fp64": native.BL_PREC_FP64,
             "fast": native.BL_PREC_FAST}
    prec = codes[args.precision]
    peaks = None if args.no_peaks else measure_peaks(native, device)
    wl = build_workload(torch, prec, device, args.case, rank, world)
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
    roofs = form_rooflines(args.precision, attempts, samples, geo_avg, tr_avg, peaks)
    work_hist = {"dp_attempts_per_ray": _hist(torch.cat([o["steps"].reshape(-1) for o in outs]).cpu().numpy()),
                 "samples_per_ray": _hist(torch.cat([o["samples"].reshape(-1) for o in outs]).cpu().numpy())}
    status_bad = sum(int(((o["status"] != 1) & (o["status"] != 2)).sum()) for o in outs)
    # the secondary measurements below allocate their own workspaces
    del ws
    torch.cuda.empty_cache()

    other, other_outs = None, {}
    if not args.no_other_forms:
        other = {}
        for name in PREC_NAMES:
            if name == args.precision:
                continue
            other[name], other_outs[name] = time_form(torch, native, images, wl, codes[name],
                                                      device, steps=3, warmup=2, peaks=peaks,
                                                      name=name)
    layout_cmp = None
    if not args.no_other_forms and GRID_LAYOUT == "cells":
        # the fast form's step on the grids in the plane layout (the layout as generated)
        wl_planes = dict(wl, gps=[wl["gp"]] * len(cams), prims=wl["prims_planes"])
        layout_cmp, _ = time_form(torch, native, images, wl_planes, native.BL_PREC_FAST, device,
                                  steps=3, warmup=2, name="fast")
    hires = hires_img = hires_host = hires_fast = hires_fast_img = None
    if not args.no_hires and args.case == "full":
        hires, hires_img, hires_host = measure_hires(torch, native, images, prec, device,
                                                     keep_image=True, keep_host=True)
        if prec != native.BL_PREC_FAST:
            hires_fast, hires_fast_img, _ = measure_hires(torch, native, images,
                                                          native.BL_PREC_FAST, device,
                                                          keep_image=True)
        else:
            hires_fast, hires_fast_img = hires, hires_img
    variants = None
    if not args.no_variants:
        variants = measure_variants(torch, native, images, wl, prec, device)
    plan = None
    if not args.no_plan:
        plan = measure_plan(torch, native, images, wl, native.BL_PREC_FAST, device)
    model = None
    if (not args.no_mlp or not args.no_slow) and args.case == "full":
        from paper_2203_15963_gb300 import coefmodel
        t0 = time.perf_counter()
        params, hist = coefmodel.train(device=device)
        torch.cuda.synchronize()
        model = (params, time.perf_counter() - t0, float(hist[-500:].mean()))
    mlp = None
    if not args.no_mlp and args.case == "full":
        mlp = measure_mlp(torch, native, images, device, hires_fast_img,
                          hires_img if prec == native.BL_PREC_FP64 else None,
                          hires if prec == native.BL_PREC_FP64 else None, *model)
    slow = None
    if not args.no_slow and args.case == "full":
        slow = measure_slow(torch, native, images, device, model[0] if model else None)
    model = None
    adaptive = None
    if not args.no_adaptive and args.case == "full":
        adaptive = measure_adaptive(torch, native, native.BL_PREC_FAST, device)
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(torch, native, wl, prec, max(1, min(args.steps, 3)))
    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the CPU-baseline leg: the oracle on a seeded pixel sample of every image, which
        # also judges each GPU form's images on those pixels
        cpu, ref = cpu_baseline(wl, args.oracle_pixels, single_thread=True)
        errors = {args.precision: oracle_image_error(outs, ref)}
        for name, o in other_outs.items():
            errors[name] = oracle_image_error(o, ref)
        ref = None
        if hires_host is not None:
            cpu["hires_sample"] = hires_oracle_sample(hires_host, hires_img, hires_fast_img,
                                                      args.oracle_pixels)
    hires_host = hires_img = hires_fast_img = None

    if rank == 0:
        roof = roofs[0]
        line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {native.BL_PREC_MIXED: "f64+f32", native.BL_PREC_FP64: "f64",
                          native.BL_PREC_FAST: "df64+f32"}[prec],
                "data": "synthetic",
                "config": workload_config(args, world),
                "kernel_ms": {"geodesic": geo_avg * 1e3, "transfer": tr_avg * 1e3},
                "work": {"dp_attempts": attempts, "samples": samples,
                         "rays_not_terminated_normally": status_bad, "per_ray": work_hist},
                "roofline": roof, "roofline_other_kernel": roofs[1], "peaks": peaks,
                "image_error_vs_oracle": errors,
                "cpu_baseline": cpu, "e2e": e2e, "other_forms": other,
                "plane_layout_fast": layout_cmp,
                "variants": variants, "plan": plan, "hires": hires, "hires_fast": hires_fast,
                "mlp": mlp, "slow_light": slow, "adaptive": adaptive,
                "gpu_launches": int(launches), "clocks": clk, "return_codes": sorted(set(rcs)),
                "kernel_source_hash": kernel_source_hash()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def time_form(torch, native, images, wl, code, device, steps, warmup, peaks=None, name=None):
    """Short CUDA-event timing of the same workload in another precision form, with its
    rooflines. Returns (line, outputs)."""
    import dataclasses
    mets = [dataclasses.replace(m, precision=code) for m in wl["mets"]]
    cams = wl["cams"]
    ws = torch.empty(native.blacklight_workspace_size(cams, mets), dtype=torch.uint8,
                     device=device)
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    outs = [images.alloc_outputs(c.n, dt, device=device, samples=True) for c in cams]
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
    line = {"value": rays / ms * 1e3, "ms_per_step": ms, "steps": steps,
            "dtype": {native.BL_PREC_MIXED: "f64+f32", native.BL_PREC_FP64: "f64",
                      native.BL_PREC_FAST: "df64+f32"}[code],
            "kernel_ms": {"geodesic": geo / steps, "transfer": tr / steps}}
    if name is not None and peaks is not None:
        attempts = sum(int(o["steps"].long().sum()) for o in outs)
        samples = sum(int(o["samples"].long().sum()) for o in outs)
        line["roofline"] = list(form_rooflines(name, attempts, samples, geo / steps / 1e3,
                                               tr / steps / 1e3, peaks))
    return line, outs


def measure_hires(torch, native, images, code, device, steps=3, warmup=2, coef_mlp=None,
                  keep_image=False, keep_host=False):
    """The metric's 1024^2 point: one 1024x1024 image (a = 0.94, i = 17 deg, 230 GHz) on the
    512x256x256 torus (1 GiB of float32), timed like the main workload. coef_mlp selects the
    learned coefficient model. Returns (line, Stokes image or None, host inputs or None)."""
    from paper_2203_15963_gb300 import synth as S
    cam, met, gp, prim = S.workload_inputs("torus512_cam1024", 0.94, 17.0)
    met = S.Metric(**{**met.__dict__, "precision": code})
    p, gpd = device_grid(torch, prim, gp, device)
    host = (cam, met, gp, prim) if keep_host else None
    del prim
    # the learned model's outputs need room beyond blacklight_workspace_size (8 floats a pool
    # record): that line lets the library size its scratch (one wave, from the stream-ordered
    # memory pool, told to keep it between calls as the end-to-end line does)
    ws = (None if coef_mlp is not None else
          torch.empty(native.blacklight_workspace_size([cam], [met]), dtype=torch.uint8,
                      device=device))
    if ws is None:
        native.blacklight_set_memory_retention(2 ** 64 - 1)
    dt = torch.float64 if code == native.BL_PREC_FP64 else torch.float32
    out = images.alloc_outputs(cam.n, dt, device=device)
    for _ in range(warmup):
        native.blacklight_trace_batch([cam], [met], [gpd], [p], [FREQ], [out], workspace=ws,
                                      coef_mlp=coef_mlp)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    geo = tr = 0.0
    e0.record()
    for _ in range(steps):
        native.blacklight_trace_batch([cam], [met], [gpd], [p], [FREQ], [out], workspace=ws,
                                      flags=native.BL_TIMING, coef_mlp=coef_mlp)
        g, t = native.blacklight_last_kernel_ms()
        geo += g
        tr += t
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    if ws is None:
        native.blacklight_set_memory_retention(0)
    bad = int(((out["status"] != 1) & (out["status"] != 2)).sum())
    del ws, p
    torch.cuda.empty_cache()
    line = {"workload": "torus512_cam1024", "value": cam.n * cam.n / ms * 1e3, "unit": "rays/s",
            "ms_per_step": ms, "steps": steps,
            "dtype": {native.BL_PREC_MIXED: "f64+f32", native.BL_PREC_FP64: "f64",
                      native.BL_PREC_FAST: "df64+f32"}[code],
            "kernel_ms": {"geodesic": geo / steps, "transfer": tr / steps},
            "rays_not_terminated_normally": bad}
    return line, (out if keep_image else None), host


def hires_oracle_sample(host, img, img_fast, n_pix, seed=7):
    """CPU-baseline leg at the 1024^2 point: the oracle on n_pix seeded pixels of the 1024^2
    image (512x256x256 torus), its rate on the host cores, and the GPU images' error against
    it on those pixels."""
    import numpy as np
    import oracle as O
    cam, met, gp, prim = host
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(cam.n * cam.n, n_pix, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    ref = O.trace(cam, met, gp, prim, FREQ, pix=pix, nthreads=0)
    dt = time.perf_counter() - t0
    out = {"value": n_pix / dt, "unit": "rays/s", "cores": os.cpu_count() or 1,
           "sample": f"{n_pix} seeded pixels of the 1024^2 image on the 512x256x256 torus"}
    if img is not None:
        out["image_error"] = oracle_image_error([img], [ref])
    if img_fast is not None and img_fast is not img:
        out["image_error_fast"] = oracle_image_error([img_fast], [ref])
    return out


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


def measure_mlp(torch, native, images, device, fast_out, out64, line64, params, train_s,
                final_loss):
    """Learned coefficients at the 1024^2 point: the model trained on the GPU (default recipe),
    then the image traced with the fused tensor-core transfer (double-float geodesics, FP32
    transfer), next to the plain FP64 form of the same image (out64/line64 when already
    measured): speedup and image error against the FP64 image, and the exact-fit fast form's
    error for comparison."""
    from paper_2203_15963_gb300 import coefmodel
    line, img, _ = measure_hires(torch, native, images, native.BL_PREC_FAST, device, steps=3,
                                 warmup=2, coef_mlp=params, keep_image=True)
    if out64 is None:
        line64, out64, _ = measure_hires(torch, native, images, native.BL_PREC_FP64, device,
                                         steps=1, warmup=1, keep_image=True)
    line.update({
        "form": "double-float geodesics, FP32 transfer, learned coefficients (BF16 tensor cores)",
        "train": {"seconds": train_s, "samples": coefmodel.N_SAMPLES, "batch": coefmodel.BATCH,
                  "steps": coefmodel.STEPS, "final_mse_normalised": final_loss},
        "fp64_form": {"value": line64["value"], "kernel_ms": line64["kernel_ms"]},
        "speedup_over_fp64_form": line["value"] / line64["value"],
        "image_rel_l2_vs_fp64_form": rel_l2(torch, img["stokes"], out64["stokes"]),
        "exact_fast_rel_l2_vs_fp64_form": (rel_l2(torch, fast_out["stokes"], out64["stokes"])
                                           if fast_out is not None else None)})
    del img
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
    import dataclasses
    from paper_2203_15963_gb300 import synth as S
    cams = wl["cams"]
    mets = [dataclasses.replace(m, precision=code) for m in wl["mets"]]
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
            "dtype": {native.BL_PREC_MIXED: "f64+f32", native.BL_PREC_FP64: "f64",
                      native.BL_PREC_FAST: "df64+f32"}[code],
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
            "value": plan_rays / plan_ms * 1e3, "unit": "rays/s", "ms_per_step": plan_ms,
            "steps": steps, "return_code": plan_rc,
            "dtype": {native.BL_PREC_MIXED: "f64+f32", native.BL_PREC_FP64: "f64",
                      native.BL_PREC_FAST: "df64+f32"}[code],
            "timing": "CUDA events around replays of the adaptive plan (every level in one "
                      "CUDA graph)",
            "rays_per_step": plan_rays, "rays_per_level": lr.sum(axis=0).tolist(),
            "direct_call": {"value": rays / sec, "ms_per_step": sec * 1e3,
                            "timing": "host wall clock of blacklight_trace_adaptive (levels "
                                      "run on the device without host round trips; one "
                                      "synchronisation at the end)"}}


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
