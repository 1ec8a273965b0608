"""Thin ctypes binding of libblacklight.so (include/blacklight.h): argument marshalling only.

Every function keeps the C name. Tensors are torch tensors on the current CUDA device; the
binding passes their data pointers and the current torch stream. There is no CPU fallback:
if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_SRC_DIR = os.path.join(_HERE, "csrc")
_LIB = os.path.join(_HERE, "_lib", "libblacklight.so")
_INCLUDE = os.path.join(_ROOT, "include")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

BL_PREC_FP64, BL_PREC_MIXED, BL_PREC_FAST = 0, 1, 2
BL_GRID_PLANES, BL_GRID_CELLS = 0, 1
BL_ASYNC = 1
BL_TIMING = 2
RAY_STATUS = {0: "ok", 1: "horizon", 2: "escaped", 3: "max_steps", 4: "underflow", 5: "nan",
              6: "overflow"}


def nvcc_command():
    return ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-I" + _INCLUDE, "-o", _LIB, os.path.join(_SRC_DIR, "bl_api.cu")]


def build(force: bool = False) -> str:
    """Compile libblacklight.so for sm_103a in-tree (skipped when up to date)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    srcs = [os.path.join(_SRC_DIR, f) for f in os.listdir(_SRC_DIR)]
    srcs.append(os.path.join(_INCLUDE, "blacklight.h"))
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(s) for s in srcs)):
        return _LIB
    subprocess.run(nvcc_command(), check=True)
    return _LIB


def library_path() -> str:
    return _LIB


class Camera(C.Structure):
    _fields_ = [("size", C.c_uint32), ("r", C.c_double), ("theta", C.c_double),
                ("phi", C.c_double), ("u_p", C.c_double * 3), ("k_p", C.c_double * 3),
                ("width", C.c_double), ("n", C.c_int32), ("psi", C.c_double),
                ("kind", C.c_int32), ("nu_at_infinity", C.c_int32)]


class Metric(C.Structure):
    _fields_ = [("size", C.c_uint32), ("mass", C.c_double), ("spin", C.c_double),
                ("r_in_over_rhor", C.c_double), ("tol_abs", C.c_double), ("tol_rel", C.c_double),
                ("ds_max", C.c_double), ("h0_frac", C.c_double), ("max_steps", C.c_int64),
                ("flat", C.c_int32), ("precision", C.c_int32), ("integrator", C.c_int32),
                ("f_step", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("size", C.c_uint32), ("prim", C.c_void_p), ("n_r", C.c_int32),
                ("n_theta", C.c_int32), ("n_phi", C.c_int32), ("r_min", C.c_double),
                ("r_max", C.c_double), ("gamma_ad", C.c_double), ("r_high", C.c_double),
                ("r_low", C.c_double), ("mu", C.c_double), ("ne_over_ni", C.c_double),
                ("sigma_cut", C.c_double), ("rho_unit_cgs", C.c_double),
                ("mass_msun", C.c_double), ("interp", C.c_int32), ("coef_mlp", C.c_void_p),
                ("n_snapshots", C.c_int32), ("time_interp", C.c_int32), ("t_first", C.c_double),
                ("dt_snapshots", C.c_double), ("t_camera", C.c_double), ("layout", C.c_int32)]


class MlpTrain(C.Structure):
    _fields_ = [("size", C.c_uint32), ("n", C.c_int64), ("inputs", C.c_void_p),
                ("targets", C.c_void_p), ("batch", C.c_int32), ("steps", C.c_int64),
                ("lr_start", C.c_double), ("lr_end", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double)]


MLP_PARAMS = 4906


class LaunchConfig(C.Structure):
    _fields_ = [("size", C.c_uint32), ("ray_order", C.c_int32), ("geo_ctas_per_sm", C.c_int32),
                ("tr_ctas_per_sm", C.c_int32), ("run_ms", C.c_float), ("ilv_block", C.c_int32)]


BL_PLAN_AUTOTUNE = 4


class Adapt(C.Structure):
    _fields_ = [("size", C.c_uint32), ("block", C.c_int32), ("max_level", C.c_int32),
                ("criterion", C.c_int32), ("threshold", C.c_double), ("min_count", C.c_int32),
                ("min_intensity", C.c_double)]


BL_CRIT_ABS_GRAD, BL_CRIT_REL_GRAD, BL_CRIT_ABS_LAPL, BL_CRIT_REL_LAPL = 0, 1, 2, 3


class Peaks(C.Structure):
    _fields_ = [("size", C.c_uint32), ("sm_count", C.c_int32), ("sm_clock_khz", C.c_int32),
                ("fp64_tflops", C.c_double), ("fp32_tflops", C.c_double),
                ("df64_tflops", C.c_double), ("probe_ms", C.c_double)]


class Out(C.Structure):
    _fields_ = [("size", C.c_uint32), ("stokes", C.c_void_p), ("dtype", C.c_int32),
                ("status", C.c_void_p), ("steps", C.c_void_p), ("end_state", C.c_void_p),
                ("samples", C.c_void_p), ("aux", C.c_void_p)]


AUX_COUNT = 26
BL_UNPOLARIZED = 8
BL_INT_DP, BL_INT_RK4, BL_INT_RK2 = 0, 1, 2


_lib = None


def load():
    """Load libblacklight.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB):
        raise RuntimeError(f"libblacklight.so is not built ({_LIB}); run __graft_entry__.build()")
    L = C.CDLL(_LIB)
    P = C.c_void_p
    L.blacklight_trace_batch.argtypes = [C.c_int32, C.POINTER(Camera), C.POINTER(Metric),
                                         C.POINTER(Grid), C.POINTER(C.c_double), C.POINTER(Out),
                                         P, C.c_size_t, P, C.c_uint32]
    L.blacklight_trace.argtypes = [C.POINTER(Camera), C.POINTER(Metric), C.POINTER(Grid),
                                   C.c_double, C.POINTER(Out), P, C.c_uint32]
    L.blacklight_trace_adaptive.argtypes = [C.c_int32, C.POINTER(Camera), C.POINTER(Metric),
                                            C.POINTER(Grid), C.POINTER(C.c_double),
                                            C.POINTER(Adapt), C.POINTER(Out),
                                            C.POINTER(C.c_int32), P]
    L.blacklight_adapt_flags.argtypes = [C.c_int64, P, C.POINTER(Adapt), P, P]
    L.blacklight_trace_noalloc.argtypes = [C.POINTER(Camera), C.POINTER(Metric), C.POINTER(Grid),
                                           C.c_double, C.POINTER(Out), P, C.c_uint32]
    L.blacklight_trace_host.argtypes = [C.POINTER(Camera), C.POINTER(Metric), C.POINTER(Grid),
                                        C.c_double, C.POINTER(Out), P]
    L.blacklight_geodesics.argtypes = [C.POINTER(Camera), C.POINTER(Metric), C.POINTER(Out), P,
                                       C.c_uint32]
    L.blacklight_grid_pack.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P]
    L.blacklight_workspace_size.argtypes = [C.c_int32, C.POINTER(Camera), C.POINTER(Metric)]
    L.blacklight_workspace_size.restype = C.c_size_t
    L.blacklight_coefficients.argtypes = [C.c_int64, P, P, C.c_int32, P]
    L.blacklight_stokes_step.argtypes = [C.c_int64, P, P, P, P, C.c_int32, P]
    L.blacklight_bessel_k.argtypes = [C.c_int64, P, P, C.c_int32, P]
    L.blacklight_mlp_init.argtypes = [P, C.c_uint64, P]
    L.blacklight_mlp_dataset.argtypes = [C.c_int64, C.c_uint64, P, P, P]
    L.blacklight_mlp_targets.argtypes = [C.c_int64, P, P, P]
    L.blacklight_mlp_normalise.argtypes = [C.c_int64, P, P, P, P]
    L.blacklight_mlp_train.argtypes = [C.POINTER(MlpTrain), P, P, P]
    L.blacklight_mlp_grad.argtypes = [P, C.c_int64, P, P, P, C.POINTER(C.c_float), P]
    L.blacklight_mlp_forward.argtypes = [P, C.c_int64, P, P, P]
    L.blacklight_mlp_coefficients.argtypes = [P, C.c_int64, P, P, P]
    L.blacklight_plan_create.argtypes = [C.c_int32, C.POINTER(Camera), C.POINTER(Metric),
                                         C.POINTER(Grid), C.POINTER(C.c_double), C.POINTER(Out),
                                         C.POINTER(LaunchConfig), C.c_uint32, P,
                                         C.POINTER(C.c_void_p)]
    L.blacklight_plan_run.argtypes = [P, P]
    L.blacklight_plan_check.argtypes = [P, P]
    L.blacklight_plan_config.argtypes = [P, C.POINTER(LaunchConfig)]
    L.blacklight_plan_destroy.argtypes = [P]
    L.blacklight_plan_create_adaptive.argtypes = [C.c_int32, C.POINTER(Camera), C.POINTER(Metric),
                                                  C.POINTER(Grid), C.POINTER(C.c_double),
                                                  C.POINTER(Adapt), C.POINTER(Out), C.c_uint32, P,
                                                  C.POINTER(C.c_void_p)]
    L.blacklight_plan_level_rays.argtypes = [P, C.POINTER(C.c_int32), P]
    L.blacklight_selftest_wait.argtypes = [C.c_int64, C.c_int32, P]
    L.blacklight_set_memory_retention.argtypes = [C.c_uint64]
    L.blacklight_measure_peaks.argtypes = [C.POINTER(Peaks), C.c_int32, P]
    L.blacklight_trace_host_batch.argtypes = [C.c_int32, C.POINTER(Camera), C.POINTER(Metric),
                                              C.POINTER(Grid), C.POINTER(C.c_double),
                                              C.POINTER(Out), P, C.c_uint32]
    L.blacklight_strerror.argtypes = [C.c_int]
    L.blacklight_strerror.restype = C.c_char_p
    L.blacklight_last_error_detail.argtypes = []
    L.blacklight_last_error_detail.restype = C.c_char_p
    L.blacklight_launch_count.argtypes = [C.c_int]
    L.blacklight_launch_count.restype = C.c_uint64
    L.blacklight_last_kernel_ms.argtypes = [C.POINTER(C.c_float)]
    _lib = L
    return L


class BlacklightError(RuntimeError):
    def __init__(self, code, detail):
        super().__init__(f"blacklight error {code}: {detail}")
        self.code = code


def _check(rc):
    if rc < 0:
        L = load()
        raise BlacklightError(rc, (L.blacklight_strerror(rc) or b"").decode() + ": "
                              + (L.blacklight_last_error_detail() or b"").decode())
    return rc


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ------------------------------- struct builders ---------------------------------------
def camera_struct(cam) -> Camera:
    return Camera(C.sizeof(Camera), cam.r, cam.theta, cam.phi, (C.c_double * 3)(*cam.u_p),
                  (C.c_double * 3)(*cam.k_p), cam.width, cam.n, cam.psi, cam.kind,
                  cam.nu_at_infinity)


def metric_struct(met, precision=None) -> Metric:
    p = met.precision if precision is None else precision
    return Metric(C.sizeof(Metric), met.mass, met.spin, met.r_in_over_rhor, met.tol_abs,
                  met.tol_rel, met.ds_max, met.h0_frac, int(met.max_steps), met.flat, p,
                  getattr(met, "integrator", 0), getattr(met, "f_step", 0.01))


def grid_struct(gp, prim_ptr, coef_mlp=None) -> Grid:
    """coef_mlp: optional tensor holding the learned coefficient model's parameters."""
    return Grid(C.sizeof(Grid), prim_ptr, gp.n_r, gp.n_theta, gp.n_phi, gp.r_min, gp.r_max,
                gp.gamma_ad, gp.r_high, gp.r_low, gp.mu, gp.ne_over_ni, gp.sigma_cut,
                gp.rho_unit_cgs, gp.mass_msun, gp.interp,
                None if coef_mlp is None else coef_mlp.data_ptr(),
                getattr(gp, "n_snapshots", 1), getattr(gp, "time_interp", 1),
                getattr(gp, "t_first", 0.0), getattr(gp, "dt_snapshots", 1.0),
                getattr(gp, "t_camera", 0.0), getattr(gp, "layout", BL_GRID_PLANES))


def out_struct(stokes=None, status=None, steps=None, end_state=None, samples=None,
               aux=None) -> Out:
    import torch
    dtype = 0
    if stokes is not None:
        dtype = 0 if stokes.dtype == torch.float64 else 1
    return Out(C.sizeof(Out), _ptr(stokes), dtype, _ptr(status), _ptr(steps), _ptr(end_state),
               _ptr(samples), _ptr(aux))


# ------------------------------------ calls ---------------------------------------------
def blacklight_trace_batch(cams, mets, gps, prims, freqs, outs, workspace=None, stream=None,
                           flags=0, coef_mlp=None):
    """cams/mets/gps: synth dataclasses; prims: CUDA float32 tensors; outs: dicts of tensors;
    coef_mlp: optional CUDA float32 tensor of the learned coefficient model (all images)."""
    L = load()
    n = len(cams)
    ca = (Camera * n)(*[camera_struct(c) for c in cams])
    ma = (Metric * n)(*[metric_struct(m) for m in mets])
    ga = (Grid * n)(*[grid_struct(g, p.data_ptr(), coef_mlp) for g, p in zip(gps, prims)])
    fa = (C.c_double * n)(*[float(f) for f in freqs])
    oa = (Out * n)(*[out_struct(**o) for o in outs])
    ws_ptr, ws_bytes = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel()
                                                           * workspace.element_size())
    return _check(L.blacklight_trace_batch(n, ca, ma, ga, fa, oa, ws_ptr, ws_bytes,
                                           _stream(stream), flags))


def blacklight_trace(cam, met, gp, prim, freq, out, stream=None, flags=0):
    L = load()
    cs, ms, gs, os_ = camera_struct(cam), metric_struct(met), grid_struct(gp, prim.data_ptr()), \
        out_struct(**out)
    return _check(L.blacklight_trace(C.byref(cs), C.byref(ms), C.byref(gs), float(freq),
                                     C.byref(os_), _stream(stream), flags))


def blacklight_trace_noalloc(cam, met, gp, prim, freq, out, stream=None, flags=0):
    """blacklight_trace without any device allocation (fixed in-library scratch, <= 1024 rays)."""
    L = load()
    cs, ms, gs, os_ = camera_struct(cam), metric_struct(met), grid_struct(gp, prim.data_ptr()), \
        out_struct(**out)
    return _check(L.blacklight_trace_noalloc(C.byref(cs), C.byref(ms), C.byref(gs), float(freq),
                                             C.byref(os_), _stream(stream), flags))


def blacklight_trace_host(cam, met, gp, prim_host, freq, out_host, stream=None, coef_mlp=None):
    """prim_host, coef_mlp (optional) and the tensors in out_host are CPU tensors (pinned for
    speed)."""
    L = load()
    cs, ms = camera_struct(cam), metric_struct(met)
    gs = grid_struct(gp, prim_host.data_ptr(), coef_mlp)
    os_ = out_struct(**out_host)
    return _check(L.blacklight_trace_host(C.byref(cs), C.byref(ms), C.byref(gs), float(freq),
                                          C.byref(os_), _stream(stream)))


def blacklight_trace_host_batch(cams, mets, gps, prims_host, freqs, outs_host, stream=None,
                                flags=0, coef_mlp=None):
    """blacklight_trace_batch with CPU tensors (pinned for speed) for grids and outputs; images
    that share a grid tensor upload it once."""
    L = load()
    n = len(cams)
    ca = (Camera * n)(*[camera_struct(c) for c in cams])
    ma = (Metric * n)(*[metric_struct(m) for m in mets])
    ga = (Grid * n)(*[grid_struct(g, p.data_ptr(), coef_mlp) for g, p in zip(gps, prims_host)])
    fa = (C.c_double * n)(*[float(f) for f in freqs])
    oa = (Out * n)(*[out_struct(**o) for o in outs_host])
    return _check(L.blacklight_trace_host_batch(n, ca, ma, ga, fa, oa, _stream(stream), flags))


def blacklight_grid_pack(planes, cells, gp, stream=None):
    """Repack the grid tensor `planes` ([snapshots][8][phi][theta][r]) into `cells`
    ([snapshots][phi][theta][r][8]), both on the device, on `stream`."""
    n_snap = max(1, getattr(gp, "n_snapshots", 1))
    want = 8 * gp.n_r * gp.n_theta * gp.n_phi * n_snap
    if planes.numel() < want or cells.numel() < want:
        raise ValueError("grid tensors smaller than the grid")
    return _check(load().blacklight_grid_pack(_ptr(planes), _ptr(cells), gp.n_r, gp.n_theta,
                                              gp.n_phi, n_snap, _stream(stream)))


def blacklight_geodesics(cam, met, out, stream=None, flags=0):
    L = load()
    cs, ms, os_ = camera_struct(cam), metric_struct(met), out_struct(**out)
    return _check(L.blacklight_geodesics(C.byref(cs), C.byref(ms), C.byref(os_),
                                         _stream(stream), flags))


def blacklight_workspace_size(cams, mets) -> int:
    L = load()
    n = len(cams)
    ca = (Camera * n)(*[camera_struct(c) for c in cams])
    ma = (Metric * n)(*[metric_struct(m) for m in mets])
    return int(L.blacklight_workspace_size(n, ca, ma))


def blacklight_coefficients(inp, out, precision, stream=None):
    return _check(load().blacklight_coefficients(inp.shape[0], _ptr(inp), _ptr(out), precision,
                                                 _stream(stream)))


def blacklight_stokes_step(coef, s0, dl, s1, precision, stream=None):
    return _check(load().blacklight_stokes_step(coef.shape[0], _ptr(coef), _ptr(s0), _ptr(dl),
                                                _ptr(s1), precision, _stream(stream)))


def blacklight_bessel_k(x, out, precision, stream=None):
    return _check(load().blacklight_bessel_k(x.shape[0], _ptr(x), _ptr(out), precision,
                                             _stream(stream)))


# ------------------------------- plans (CUDA-graph replay) ------------------------------
class Plan:
    """A batched trace captured once in a CUDA graph (blacklight_plan_*). Keeps references to
    the tensors whose pointers the plan binds."""

    def __init__(self, cams, mets, gps, prims, freqs, outs, autotune=False, config=None,
                 stream=None, coef_mlp=None):
        L = load()
        n = len(cams)
        ca = (Camera * n)(*[camera_struct(c) for c in cams])
        ma = (Metric * n)(*[metric_struct(m) for m in mets])
        ga = (Grid * n)(*[grid_struct(g, p.data_ptr(), coef_mlp) for g, p in zip(gps, prims)])
        fa = (C.c_double * n)(*[float(f) for f in freqs])
        oa = (Out * n)(*[out_struct(**o) for o in outs])
        cfg = None
        if config is not None:
            cfg = LaunchConfig(C.sizeof(LaunchConfig), int(config.get("ray_order", 0)),
                               int(config.get("geo_ctas_per_sm", 0)),
                               int(config.get("tr_ctas_per_sm", 0)), 0.0,
                               int(config.get("ilv_block", 0)))
        h = C.c_void_p()
        _check(L.blacklight_plan_create(n, ca, ma, ga, fa, oa,
                                        None if cfg is None else C.byref(cfg),
                                        BL_PLAN_AUTOTUNE if autotune else 0, _stream(stream),
                                        C.byref(h)))
        self._h = h
        self._keep = (list(prims), list(outs), coef_mlp)

    def run(self, stream=None):
        return _check(load().blacklight_plan_run(self._h, _stream(stream)))

    def check(self, stream=None):
        return _check(load().blacklight_plan_check(self._h, _stream(stream)))

    def config(self):
        c = LaunchConfig(C.sizeof(LaunchConfig), 0, 0, 0, 0.0, 0)
        _check(load().blacklight_plan_config(self._h, C.byref(c)))
        return {"ray_order": c.ray_order, "geo_ctas_per_sm": c.geo_ctas_per_sm,
                "tr_ctas_per_sm": c.tr_ctas_per_sm, "run_ms": c.run_ms,
                "ilv_block": c.ilv_block}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().blacklight_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdaptivePlan(Plan):
    """An adaptive trace (blacklight_plan_create_adaptive) replayed as one CUDA graph."""

    def __init__(self, cams, mets, gps, prims, freqs, adapt, outs, flags=0, stream=None,
                 coef_mlp=None):
        L = load()
        n = len(cams)
        ca = (Camera * n)(*[camera_struct(c) for c in cams])
        ma = (Metric * n)(*[metric_struct(m) for m in mets])
        ga = (Grid * n)(*[grid_struct(g, p.data_ptr(), coef_mlp) for g, p in zip(gps, prims)])
        fa = (C.c_double * n)(*[float(f) for f in freqs])
        oa = (Out * n)(*[out_struct(**o) for o in outs])
        h = C.c_void_p()
        _check(L.blacklight_plan_create_adaptive(n, ca, ma, ga, fa, C.byref(adapt), oa, flags,
                                                 _stream(stream), C.byref(h)))
        self._h = h
        self._keep = (list(prims), list(outs), coef_mlp)
        self._shape = (n, adapt.max_level + 1)

    def level_rays(self, stream=None):
        import numpy as np
        lr = np.zeros(self._shape, dtype=np.int32)
        _check(load().blacklight_plan_level_rays(self._h, lr.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 _stream(stream)))
        return lr


# ------------------------------- learned coefficient model ------------------------------
def blacklight_mlp_init(params, seed, stream=None):
    return _check(load().blacklight_mlp_init(_ptr(params), int(seed), _stream(stream)))


def blacklight_mlp_dataset(n, seed, inputs, targets, stream=None):
    return _check(load().blacklight_mlp_dataset(int(n), int(seed), _ptr(inputs), _ptr(targets),
                                                _stream(stream)))


def blacklight_mlp_targets(inputs, targets, stream=None):
    return _check(load().blacklight_mlp_targets(inputs.shape[0], _ptr(inputs), _ptr(targets),
                                                _stream(stream)))


def blacklight_mlp_normalise(inputs, targets, params, stream=None):
    return _check(load().blacklight_mlp_normalise(targets.shape[0], _ptr(inputs), _ptr(targets),
                                                  _ptr(params), _stream(stream)))


def blacklight_mlp_train(params, inputs, targets, batch, steps, lr_start, lr_end, beta1=0.9,
                         beta2=0.999, eps=1e-8, loss_history=None, stream=None):
    cfg = MlpTrain(C.sizeof(MlpTrain), inputs.shape[0], inputs.data_ptr(), targets.data_ptr(),
                   int(batch), int(steps), float(lr_start), float(lr_end), float(beta1),
                   float(beta2), float(eps))
    return _check(load().blacklight_mlp_train(C.byref(cfg), _ptr(params), _ptr(loss_history),
                                              _stream(stream)))


def blacklight_mlp_grad(params, inputs, targets, grad, stream=None) -> float:
    loss = C.c_float(0.0)
    _check(load().blacklight_mlp_grad(_ptr(params), inputs.shape[0], _ptr(inputs), _ptr(targets),
                                      _ptr(grad), C.byref(loss), _stream(stream)))
    return float(loss.value)


def blacklight_mlp_forward(params, inputs, outputs, stream=None):
    return _check(load().blacklight_mlp_forward(_ptr(params), inputs.shape[0], _ptr(inputs),
                                                _ptr(outputs), _stream(stream)))


def blacklight_mlp_coefficients(params, inp, out, stream=None):
    return _check(load().blacklight_mlp_coefficients(_ptr(params), inp.shape[0], _ptr(inp),
                                                     _ptr(out), _stream(stream)))


BL_ETIMEOUT = -5


def blacklight_set_memory_retention(nbytes) -> int:
    return _check(load().blacklight_set_memory_retention(int(nbytes)))


def blacklight_measure_peaks(reps=5, stream=None) -> dict:
    """Measured FP64, FP32 and double-float multiply-add throughput of the current device
    (TFLOP/s, best of `reps` launches) with its SM count and maximum SM clock."""
    p = Peaks(size=C.sizeof(Peaks))
    _check(load().blacklight_measure_peaks(C.byref(p), int(reps), _stream(stream)))
    return {k: getattr(p, k) for k, _ in Peaks._fields_ if k != "size"}


def blacklight_selftest_wait(max_cycles, arrive, stream=None) -> int:
    """0 if the wait completed; BL_ETIMEOUT (returned, not raised) if it ran out."""
    rc = load().blacklight_selftest_wait(int(max_cycles), int(arrive), _stream(stream))
    if rc == BL_ETIMEOUT:
        return rc
    return _check(rc)


def blacklight_launch_count(reset=False) -> int:
    return int(load().blacklight_launch_count(1 if reset else 0))


def blacklight_last_kernel_ms():
    """(geodesic_ms, transfer_ms) of this thread's last call made with BL_TIMING."""
    ms = (C.c_float * 2)()
    _check(load().blacklight_last_kernel_ms(ms))
    return float(ms[0]), float(ms[1])


def adapt_struct(block, max_level, criterion, threshold, min_count, min_intensity=0.0) -> Adapt:
    return Adapt(C.sizeof(Adapt), block, max_level, criterion, float(threshold), min_count,
                 float(min_intensity))


def blacklight_trace_adaptive(cams, mets, gps, prims, freqs, adapt, outs, stream=None,
                              coef_mlp=None):
    """Adaptive tracing; outs[q]["stokes"] is the [4][nf][nf] composite. Returns (rc, rays per
    level [n_images][max_level + 1])."""
    import numpy as np
    L = load()
    n = len(cams)
    ca = (Camera * n)(*[camera_struct(c) for c in cams])
    ma = (Metric * n)(*[metric_struct(m) for m in mets])
    ga = (Grid * n)(*[grid_struct(g, p.data_ptr(), coef_mlp) for g, p in zip(gps, prims)])
    fa = (C.c_double * n)(*[float(f) for f in freqs])
    oa = (Out * n)(*[out_struct(**o) for o in outs])
    lr = np.zeros((n, adapt.max_level + 1), dtype=np.int32)
    rc = _check(L.blacklight_trace_adaptive(n, ca, ma, ga, fa, C.byref(adapt), oa,
                                            lr.ctypes.data_as(C.POINTER(C.c_int32)),
                                            _stream(stream)))
    return rc, lr


def blacklight_adapt_flags(I, adapt, flags, stream=None):
    return _check(load().blacklight_adapt_flags(I.shape[0], _ptr(I), C.byref(adapt), _ptr(flags),
                                                _stream(stream)))
