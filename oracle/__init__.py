"""CPU FP64 oracle for the Blacklight hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. It shares no code with the CUDA library and the CUDA path never calls it.
``build()`` compiles ``liboracle.so`` from the C++ sources next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["geometry.cpp", "radiation.cpp"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build_command():
    return (["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB_PATH]
            + [os.path.join(_HERE, s) for s in _SRC] + ["-lpthread"])


def build(force: bool = False) -> str:
    """Compile the oracle (plain C++17, no GPU) if missing or stale."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRC + ["oracle.h", "oracle_internal.hpp"]]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    subprocess.run(build_command(), check=True)
    return _LIB_PATH


class Camera(C.Structure):
    _fields_ = [("r", C.c_double), ("theta", C.c_double), ("phi", C.c_double),
                ("u_p", C.c_double * 3), ("k_p", C.c_double * 3), ("width", C.c_double),
                ("n", C.c_int32), ("psi", C.c_double), ("kind", C.c_int32),
                ("nu_at_infinity", C.c_int32)]


class Metric(C.Structure):
    _fields_ = [("mass", C.c_double), ("spin", C.c_double), ("r_in_over_rhor", C.c_double),
                ("tol_abs", C.c_double), ("tol_rel", C.c_double), ("ds_max", C.c_double),
                ("h0_frac", C.c_double), ("max_steps", C.c_int64), ("flat", C.c_int32),
                ("integrator", C.c_int32), ("f_step", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("prim", C.POINTER(C.c_float)), ("n_r", C.c_int32), ("n_theta", C.c_int32),
                ("n_phi", C.c_int32), ("r_min", C.c_double), ("r_max", C.c_double),
                ("gamma_ad", C.c_double), ("r_high", C.c_double), ("r_low", C.c_double),
                ("mu", C.c_double), ("ne_over_ni", C.c_double), ("sigma_cut", C.c_double),
                ("rho_unit_cgs", C.c_double), ("mass_msun", C.c_double), ("interp", C.c_int32),
                ("n_snapshots", C.c_int32), ("time_interp", C.c_int32), ("t_first", C.c_double),
                ("dt", C.c_double), ("t_camera", C.c_double)]


STATUS = {0: "ok", 1: "horizon", 2: "escaped", 3: "max_steps", 4: "underflow", 5: "nan"}

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.ora_metric_cks.argtypes = [_D, C.c_double, C.c_double, C.c_int, _D, _D]
        L.ora_metric_sks.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _D]
        L.ora_christoffel.argtypes = [_D, C.c_double, C.c_double, C.c_int, _D]
        L.ora_geodesic_rhs.argtypes = [_D, C.c_double, C.c_double, C.c_int, _D]
        L.ora_set_rhs_perturbation.argtypes = [C.c_int32]
        L.ora_dp_tableau.argtypes = [_D] * 5
        L.ora_r_of_x.argtypes = [_D, C.c_double]
        L.ora_r_of_x.restype = C.c_double
        L.ora_camera_pixel.argtypes = [C.POINTER(Camera), C.POINTER(Metric), C.c_int32,
                                       C.c_int32, _D, _D, _D, _D, _D]
        L.ora_geodesic.argtypes = [C.POINTER(Metric), C.c_double, _D, _D, _I64, _I64, _D,
                                   C.c_int64, _I64]
        L.ora_geodesic.restype = C.c_int32
        L.ora_sample_grid.argtypes = [C.POINTER(Grid), C.c_double, _D, _D]
        L.ora_sample_grid.restype = C.c_int32
        L.ora_plasma.argtypes = [C.POINTER(Grid), C.POINTER(Metric), _D, _D, _D, _D, _D, _D]
        L.ora_plasma.restype = C.c_int32
        L.ora_bessel_kx.argtypes = [C.c_double, C.c_double]
        L.ora_bessel_kx.restype = C.c_double
        L.ora_coefficients.argtypes = [C.c_double] * 5 + [_D]
        L.ora_stokes_step.argtypes = [_D, _D, C.c_double, _D]
        L.ora_transport_step.argtypes = [C.POINTER(Metric), _D, _D, _D, _D, C.c_double, _D, _D]
        L.ora_ray_samples.argtypes = [C.POINTER(Metric), C.POINTER(Grid), C.c_double, _D,
                                      C.c_int64, _D]
        L.ora_ray_samples.restype = C.c_int64
        L.ora_fluid_frame.argtypes = [_D] * 6
        L.ora_n_to_s.argtypes = [_D] * 6
        L.ora_s_to_n.argtypes = [_D] * 5
        L.ora_trace.argtypes = [C.POINTER(Camera), C.POINTER(Metric), C.POINTER(Grid), C.c_double,
                                C.c_int64, C.POINTER(C.c_int32), C.c_int32, _D,
                                C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64), _D, C.c_int32, _D]
        L.ora_unpolarized_step.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.ora_unpolarized_step.restype = C.c_double
        _lib = L
    return _lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _f64(n):
    return np.zeros(n, dtype=np.float64)


# --------------------------- conversions from synth dataclasses ---------------------------
def camera_struct(cam) -> Camera:
    return Camera(cam.r, cam.theta, cam.phi, (C.c_double * 3)(*cam.u_p),
                  (C.c_double * 3)(*cam.k_p), cam.width, cam.n, cam.psi, cam.kind,
                  cam.nu_at_infinity)


def metric_struct(met) -> Metric:
    return Metric(met.mass, met.spin, met.r_in_over_rhor, met.tol_abs, met.tol_rel, met.ds_max,
                  met.h0_frac, int(met.max_steps), met.flat, getattr(met, "integrator", 0),
                  getattr(met, "f_step", 0.01))


def grid_struct(gp, prim: np.ndarray) -> Grid:
    """prim: [8][n_phi][n_theta][n_r], or [n_snapshots][8][...] with gp.n_snapshots > 1."""
    assert prim.dtype == np.float32 and prim.flags.c_contiguous
    ns = getattr(gp, "n_snapshots", 1)
    assert prim.size == max(ns, 1) * 8 * gp.n_phi * gp.n_theta * gp.n_r
    return Grid(_p(prim, C.c_float), gp.n_r, gp.n_theta, gp.n_phi, gp.r_min, gp.r_max,
                gp.gamma_ad, gp.r_high, gp.r_low, gp.mu, gp.ne_over_ni, gp.sigma_cut,
                gp.rho_unit_cgs, gp.mass_msun, gp.interp, ns, getattr(gp, "time_interp", 1),
                getattr(gp, "t_first", 0.0), getattr(gp, "dt_snapshots", 1.0),
                getattr(gp, "t_camera", 0.0))


# ------------------------------------ wrappers ------------------------------------------
def metric_cks(x, mass, spin, flat=0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    glo, ghi = _f64(16), _f64(16)
    lib().ora_metric_cks(_p(x), mass, spin, flat, _p(glo), _p(ghi))
    return glo.reshape(4, 4), ghi.reshape(4, 4)


def metric_sks(r, theta, mass, spin):
    g = _f64(16)
    lib().ora_metric_sks(r, theta, mass, spin, _p(g))
    return g.reshape(4, 4)


def christoffel(x, mass, spin, flat=0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = _f64(64)
    lib().ora_christoffel(_p(x), mass, spin, flat, _p(g))
    return g.reshape(4, 4, 4)


def set_rhs_perturbation(ulps: int) -> None:
    """Test knob: component i of every later oracle geodesic right-hand side is scaled by
    (1 + (-1)^i ulps 2^-52); 0 switches it off."""
    lib().ora_set_rhs_perturbation(int(ulps))


def geodesic_rhs(y, mass, spin, flat=0):
    y = np.ascontiguousarray(y, dtype=np.float64)
    dy = _f64(8)
    lib().ora_geodesic_rhs(_p(y), mass, spin, flat, _p(dy))
    return dy


def dp_tableau():
    a, b5, b4, bm, c = _f64(49), _f64(7), _f64(7), _f64(7), _f64(7)
    lib().ora_dp_tableau(_p(a), _p(b5), _p(b4), _p(bm), _p(c))
    return a.reshape(7, 7), b5, b4, bm, c


def r_of_x(x, spin):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().ora_r_of_x(_p(x), spin)


def camera_pixel(cam, met, i, j):
    cs, ms = camera_struct(cam), metric_struct(met)
    x, k, h, v, n = _f64(4), _f64(4), _f64(4), _f64(4), _f64(1)
    lib().ora_camera_pixel(C.byref(cs), C.byref(ms), i, j, _p(x), _p(k), _p(h), _p(v), _p(n))
    return x, k, h, v, float(n[0])


def geodesic(met, r_cam, y0, max_path=0):
    ms = metric_struct(met)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    yf = _f64(8)
    att, acc, npath = (C.c_int64(), C.c_int64(), C.c_int64())
    path = _f64(8 * max_path) if max_path else None
    st = lib().ora_geodesic(C.byref(ms), r_cam, _p(y0), _p(yf), C.byref(att), C.byref(acc),
                            _p(path) if path is not None else None, max_path, C.byref(npath))
    out = dict(status=int(st), end=yf, attempts=att.value, accepted=acc.value)
    if path is not None:
        out["path"] = path[: 8 * npath.value].reshape(-1, 8)
    return out


def sample_grid(gp, prim, spin, x):
    gs = grid_struct(gp, prim)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = _f64(8)
    ok = lib().ora_sample_grid(C.byref(gs), spin, _p(x), _p(out))
    return bool(ok), out


def plasma(gp, prim, met, x):
    gs, ms = grid_struct(gp, prim), metric_struct(met)
    x = np.ascontiguousarray(x, dtype=np.float64)
    u, b, ne, te, bg = _f64(4), _f64(4), _f64(1), _f64(1), _f64(1)
    ok = lib().ora_plasma(C.byref(gs), C.byref(ms), _p(x), _p(u), _p(b), _p(ne), _p(te), _p(bg))
    return bool(ok), dict(u=u, b=b, ne=float(ne[0]), theta_e=float(te[0]), b_gauss=float(bg[0]))


def bessel_kx(nu, x):
    return lib().ora_bessel_kx(float(nu), float(x))


def coefficients(ne, theta_e, b_gauss, nu, cos_theta):
    out = _f64(8)
    lib().ora_coefficients(ne, theta_e, b_gauss, nu, cos_theta, _p(out))
    return out


def stokes_step(coef, s0, dlam):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    s0 = np.ascontiguousarray(s0, dtype=np.float64)
    s1 = _f64(4)
    lib().ora_stokes_step(_p(coef), _p(s0), dlam, _p(s1))
    return s1


def transport_step(met, x0, k0, x1, k1, h, n_re, n_im):
    ms = metric_struct(met)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x0, k0, x1, k1)]
    nre = np.ascontiguousarray(n_re, dtype=np.float64).reshape(16).copy()
    nim = np.ascontiguousarray(n_im, dtype=np.float64).reshape(16).copy()
    lib().ora_transport_step(C.byref(ms), *[_p(v) for v in a], h, _p(nre), _p(nim))
    return nre.reshape(4, 4), nim.reshape(4, 4)


def ray_samples(met, gp, prim, r_cam, y0, max_out=100000):
    """Samples of one ray, camera side first: dict of x, k, node_x, node_k, dl arrays."""
    ms, gs = metric_struct(met), grid_struct(gp, prim)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    out = _f64(17 * max_out)
    n = lib().ora_ray_samples(C.byref(ms), C.byref(gs), r_cam, _p(y0), max_out, _p(out))
    o = out[: 17 * min(n, max_out)].reshape(-1, 17)
    return dict(x=o[:, 0:4], k=o[:, 4:8], node_x=o[:, 8:12], node_k=o[:, 12:16], dl=o[:, 16])


def fluid_frame(glo, u, kup, b):
    arr = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1) for v in (glo, u, kup, b)]
    e1, e2 = _f64(4), _f64(4)
    lib().ora_fluid_frame(*[_p(v) for v in arr], _p(e1), _p(e2))
    return e1, e2


def n_to_s(glo, e1, e2, n_re, n_im):
    arr = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1) for v in (glo, e1, e2, n_re, n_im)]
    s = _f64(4)
    lib().ora_n_to_s(*[_p(v) for v in arr], _p(s))
    return s


def s_to_n(e1, e2, s):
    arr = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1) for v in (e1, e2, s)]
    nre, nim = _f64(16), _f64(16)
    lib().ora_s_to_n(*[_p(v) for v in arr], _p(nre), _p(nim))
    return nre.reshape(4, 4), nim.reshape(4, 4)


AUX_COUNT = 26


def unpolarized_step(j, alpha, dl, i0):
    return lib().ora_unpolarized_step(float(j), float(alpha), float(dl), float(i0))


def trace(cam, met, gp, prim, freq, pix=None, nthreads=0, unpolarized=False, aux=False):
    """Trace pixels (flat indices j*n+i; default all). Returns a dict of numpy arrays; with
    unpolarized=True the transfer is Eq. unpolarized (Stokes I only); with aux=True the dict
    also holds the auxiliary images, aux [n][26]."""
    cs, ms, gs = camera_struct(cam), metric_struct(met), grid_struct(gp, prim)
    if pix is None:
        pix = np.arange(cam.n * cam.n, dtype=np.int32)
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    n = pix.size
    st = _f64(4 * n)
    end = _f64(8 * n)
    status = np.zeros(n, dtype=np.int32)
    att = np.zeros(n, dtype=np.int64)
    acc = np.zeros(n, dtype=np.int64)
    smp = np.zeros(n, dtype=np.int64)
    ax = _f64(AUX_COUNT * n) if aux else None
    lib().ora_trace(C.byref(cs), C.byref(ms), C.byref(gs), float(freq), n, _p(pix, C.c_int32),
                    int(nthreads), _p(st), _p(status, C.c_int32), _p(att, C.c_int64),
                    _p(acc, C.c_int64), _p(smp, C.c_int64), _p(end), 1 if unpolarized else 0,
                    _p(ax) if aux else None)
    out = dict(stokes=st.reshape(n, 4), end=end.reshape(n, 8), status=status, attempts=att,
               accepted=acc, samples=smp, pix=pix)
    if aux:
        out["aux"] = ax.reshape(n, AUX_COUNT)
    return out


def os_cores() -> int:
    return os.cpu_count() or 1
