"""Seeded synthetic inputs: the GRMHD-like torus, camera and integrator settings.

This module only builds inputs. It holds none of the ray-tracing method's arithmetic
(geodesics, sampling, coefficients, transfer); both the CUDA path and the CPU oracle
receive exactly the arrays it returns.

Grid (spherical Kerr-Schild, Sec. 2, "Sampling"): float32 primitives stored
structure-of-arrays as ``prim[8][n_phi][n_theta][n_r]`` (r fastest) in the order
rho, u_gas, u^p_r, u^p_theta, u^p_phi, B^r, B^theta, B^phi, where u^p are the
normal-frame velocity components of Sec. 2 and B^i the coordinate magnetic-field
components. r faces are log-spaced on [r_min, r_max] with cells centred at the
log-midpoints; theta faces uniform on [0, pi]; phi faces uniform on [0, 2 pi).

Torus recipe (all seeded):
  rho    = exp(-(r-12)^2/32) * exp(-cos^2(theta)/0.18) * (1 + 0.1 N(0,1)), clamped >= 0,
           N(0,1) from numpy PCG64 default_rng(seed) drawn in C order over [phi][theta][r]
  u_gas  = 0.3 * rho * 6 / r
  u      = Keplerian: u^r = u^theta = 0, u^phi = Omega u^t, Omega = 1/(r^1.5 + a);
           cells where that orbit is not timelike get the normal observer (u^p = 0)
  B      = poloidal field from A_phi = max(rho_smooth - 0.2, 0) on cell corners
           (noise-free rho), B^r = d_theta A / sqrt(-g), B^theta = -d_r A / sqrt(-g),
           scaled so that max(p) / max(b^2/2) = 10 (p = (gamma_ad - 1) u_gas).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_PRIM = 8
BASE_SEED = 20220329


@dataclasses.dataclass
class Camera:
    """Camera centre and image plane (Sec. 2.1). Defaults: plane-parallel, static far camera."""
    r: float = 1000.0
    theta: float = math.radians(17.0)
    phi: float = 0.0
    u_p: tuple = (0.0, 0.0, 0.0)   # normal-frame velocity of the camera centre (SKS)
    k_p: tuple = (1.0, 0.0, 0.0)   # received momentum direction, covariant SKS k_i
    width: float = 40.0
    n: int = 32
    psi: float = 0.0
    kind: int = 0                  # 0 = plane-parallel (the only kind built)
    nu_at_infinity: int = 1        # frequency normalised at infinity (Sec. 2.1)


@dataclasses.dataclass
class Metric:
    """Spacetime and integrator controls (Sec. 2.2)."""
    mass: float = 1.0
    spin: float = 0.9
    r_in_over_rhor: float = 1.01
    tol_abs: float = 1e-8
    tol_rel: float = 1e-8
    ds_max: float = 0.5
    h0_frac: float = 0.01
    max_steps: int = 100000
    flat: int = 0
    precision: int = 0             # 0 = FP64 path, 1 = mixed (FP64 geodesics, FP32 transfer)
    integrator: int = 0            # 0 = DP RK5(4), 1 = RK4, 2 = RK2 (Sec. 2.2)
    f_step: float = 0.01           # RK2/RK4 step -f_step (r - r_hor) (Eq. rk_step)


@dataclasses.dataclass
class GridParams:
    """Grid geometry and plasma model constants (Secs. 2.4-2.5)."""
    n_r: int = 64
    n_theta: int = 32
    n_phi: int = 32
    r_min: float = 1.2
    r_max: float = 50.0
    gamma_ad: float = 13.0 / 9.0
    r_high: float = 20.0
    r_low: float = 1.0
    mu: float = 0.5
    ne_over_ni: float = 1.0
    sigma_cut: float = 1.0
    rho_unit_cgs: float = 1e-17
    mass_msun: float = 4.152e6
    interp: int = 1                # 1 = trilinear, 0 = nearest
    # slow light (Sec. 4): n_snapshots grids at t_first + s dt_snapshots, camera at t_camera
    n_snapshots: int = 1
    time_interp: int = 1           # 1 = linear in time, 0 = nearest snapshot
    t_first: float = 0.0
    dt_snapshots: float = 1.0
    t_camera: float = 0.0
    layout: int = 0                # memory order of prim: 0 planes [8][phi][theta][r], 1 cells


def r_faces(gp: GridParams) -> np.ndarray:
    i = np.arange(gp.n_r + 1, dtype=np.float64)
    return gp.r_min * (gp.r_max / gp.r_min) ** (i / gp.n_r)


def r_centres(gp: GridParams) -> np.ndarray:
    i = np.arange(gp.n_r, dtype=np.float64) + 0.5
    return gp.r_min * (gp.r_max / gp.r_min) ** (i / gp.n_r)


def theta_faces(gp: GridParams) -> np.ndarray:
    return np.linspace(0.0, math.pi, gp.n_theta + 1)


def theta_centres(gp: GridParams) -> np.ndarray:
    return (np.arange(gp.n_theta) + 0.5) * (math.pi / gp.n_theta)


def phi_centres(gp: GridParams) -> np.ndarray:
    return (np.arange(gp.n_phi) + 0.5) * (2.0 * math.pi / gp.n_phi)


def _sks_pieces(r, th, a, m=1.0):
    cth, sth = np.cos(th), np.sin(th)
    sigma = r * r + a * a * cth * cth
    f = 2.0 * m * r / sigma
    s2 = sth * sth
    g = {
        "tt": -(1.0 - f), "tr": f, "tph": -a * f * s2,
        "rr": 1.0 + f, "rph": -a * (1.0 + f) * s2,
        "thth": sigma, "phph": (r * r + a * a + a * a * f * s2) * s2,
    }
    return f, g


def make_torus(gp: GridParams, spin: float, seed: int, noise: float = 0.1,
               mass: float = 1.0) -> np.ndarray:
    """Return float32 prim[8][n_phi][n_theta][n_r] for the synthetic torus.

    Everything but the density noise is axisymmetric, so it is computed on the (theta, r)
    plane and broadcast over phi."""
    a = float(spin)
    rc = r_centres(gp)[None, :]                       # [1][n_r]
    thc = theta_centres(gp)[:, None]                  # [n_theta][1]
    rho_s = np.exp(-(rc - 12.0) ** 2 / 32.0) * np.exp(-np.cos(thc) ** 2 / 0.18)   # [th][r]
    rng = np.random.default_rng(seed)
    shape = (gp.n_phi, gp.n_theta, gp.n_r)
    prim = np.empty((N_PRIM,) + shape, dtype=np.float32)
    # rho and u_gas with the seeded noise (3-D), slab by slab to bound memory
    pmax = 0.0
    for k in range(gp.n_phi):
        eps = rng.standard_normal((gp.n_theta, gp.n_r))
        rho = np.maximum(rho_s * (1.0 + noise * eps), 0.0)
        ugas = 0.3 * rho * 6.0 / rc
        prim[0, k] = rho
        prim[1, k] = ugas
        pmax = max(pmax, float(((gp.gamma_ad - 1.0) * ugas).max()))

    # Keplerian velocity stored as SKS normal-frame components u^p (axisymmetric).
    r2 = np.broadcast_to(rc, rho_s.shape)
    th2 = np.broadcast_to(thc, rho_s.shape)
    f, g = _sks_pieces(r2, th2, a, mass)
    omega = 1.0 / (r2 ** 1.5 + a)
    norm = -(g["tt"] + 2.0 * omega * g["tph"] + omega * omega * g["phph"])
    ok = norm > 0.0
    ut = np.where(ok, 1.0 / np.sqrt(np.where(ok, norm, 1.0)), 0.0)
    up_r = np.where(ok, f / (1.0 + f) * ut, 0.0)
    up_th = np.zeros_like(up_r)
    up_ph = np.where(ok, omega * ut, 0.0)

    # Poloidal field from a corner-centred vector potential (noise-free density).
    rf = r_faces(gp)[None, :]
    thf = theta_faces(gp)[:, None]
    rho_corner = np.exp(-(rf - 12.0) ** 2 / 32.0) * np.exp(-np.cos(thf) ** 2 / 0.18)
    aphi = np.maximum(rho_corner - 0.2, 0.0)          # [n_theta+1][n_r+1]
    dth = math.pi / gp.n_theta
    dr = np.diff(r_faces(gp))[None, :]
    d_th = 0.5 * ((aphi[1:, :-1] - aphi[:-1, :-1]) + (aphi[1:, 1:] - aphi[:-1, 1:])) / dth
    d_r = 0.5 * ((aphi[:-1, 1:] - aphi[:-1, :-1]) + (aphi[1:, 1:] - aphi[1:, :-1])) / dr
    sqrtg = (rc ** 2 + a * a * np.cos(thc) ** 2) * np.sin(thc)
    br = d_th / sqrtg
    bth = -d_r / sqrtg
    bph = np.zeros_like(br)

    # Scale to plasma beta = 10 in the sense max(p) / max(b^2/2) = 10.
    gam = np.sqrt(1.0 + g["rr"] * up_r ** 2 + 2.0 * g["rph"] * up_r * up_ph
                  + g["thth"] * up_th ** 2 + g["phph"] * up_ph ** 2)
    u_t = gam * np.sqrt(1.0 + f)
    u_r = up_r - f / (1.0 + f) * u_t
    u_th, u_ph = up_th, up_ph
    low_r = g["tr"] * u_t + g["rr"] * u_r + g["rph"] * u_ph
    low_th = g["thth"] * u_th
    low_ph = g["tph"] * u_t + g["rph"] * u_r + g["phph"] * u_ph
    b_t = br * low_r + bth * low_th + bph * low_ph
    b_r = (br + b_t * u_r) / u_t
    b_th = (bth + b_t * u_th) / u_t
    b_ph = (bph + b_t * u_ph) / u_t
    bsq = (g["tt"] * b_t ** 2 + 2 * g["tr"] * b_t * b_r + 2 * g["tph"] * b_t * b_ph
           + g["rr"] * b_r ** 2 + 2 * g["rph"] * b_r * b_ph + g["thth"] * b_th ** 2
           + g["phph"] * b_ph ** 2)
    scale = math.sqrt(pmax / (10.0 * max(0.5 * bsq.max(), 1e-300)))

    prim[2] = up_r[None]
    prim[3] = up_th[None]
    prim[4] = up_ph[None]
    prim[5] = (br * scale)[None]
    prim[6] = (bth * scale)[None]
    prim[7] = (bph * scale)[None]
    return prim


def make_torus_series(gp: GridParams, spin: float, seed: int, n_snapshots: int, dt: float,
                      noise: float = 0.1, mass: float = 1.0) -> np.ndarray:
    """float32 [n_snapshots][8][n_phi][n_theta][n_r]: the torus of make_torus whose density
    (and internal energy) noise is carried around by the Keplerian flow, snapshot s showing it
    rotated by Omega(r) s dt, Omega = 1/(r^1.5 + a), rounded to whole cells in phi per radial
    shell. The smooth parts (velocity, field) are axisymmetric and the same in every snapshot."""
    base = make_torus(gp, spin, seed, noise, mass)
    out = np.empty((n_snapshots,) + base.shape, dtype=np.float32)
    rc = r_centres(gp)
    omega = 1.0 / (rc ** 1.5 + spin)
    dph = 2.0 * math.pi / gp.n_phi
    k = np.arange(gp.n_phi)
    for s in range(n_snapshots):
        out[s] = base
        shift = np.rint(omega * s * dt / dph).astype(np.int64)           # [n_r]
        src = (k[:, None] - shift[None, :]) % gp.n_phi                  # [n_phi][n_r]
        ridx = np.arange(gp.n_r)[None, :]
        for v in (0, 1):
            f = base[v]                                                  # [phi][theta][r]
            out[s, v] = f[src[:, None, :].repeat(gp.n_theta, 1),
                          np.arange(gp.n_theta)[None, :, None], ridx[:, None, :]]
    return out


def grid_params_for(n_r: int, n_theta: int, n_phi: int) -> GridParams:
    return GridParams(n_r=n_r, n_theta=n_theta, n_phi=n_phi)


# Named workloads (image configurations); sizes follow the paper's performance setting
# (Sec. 5) scaled to the synthetic torus.
WORKLOADS = {
    # 32x32 camera, 64x32x32 grid, a = 0.9, i = 17 deg, 230 GHz, FP64
    "torus64_cam32": dict(grid=(64, 32, 32), n=32, spins=(0.9,), incs=(17.0,),
                          freqs=(230e9,), seed_index=0),
    # 256x256 camera, 256x128x128 grid, 3 spins x 3 inclinations
    "torus256_cam256": dict(grid=(256, 128, 128), n=256, spins=(0.0, 0.5, 0.94),
                            incs=(17.0, 60.0, 90.0), freqs=(230e9,), seed_index=1),
    # 1024x1024 camera, 512x256x256 grid (1 GiB of float32), a = 0.94, 230 GHz
    "torus512_cam1024": dict(grid=(512, 256, 256), n=1024, spins=(0.94,), incs=(17.0,),
                             freqs=(230e9,), seed_index=3),
    # slow light: 8 snapshots 10 M apart of the 256x128x128 torus, 512x512 camera, a = 0.94,
    # i = 60 deg, 230 GHz, camera time 1035 M (samples near r ~ 10-20 M fall inside the span)
    "torus256_slow8_cam512": dict(grid=(256, 128, 128), n=512, spins=(0.94,), incs=(60.0,),
                                  freqs=(230e9,), seed_index=4, snapshots=8, dt=10.0,
                                  t_camera=1035.0),
    # small slow-light parity case: 4 snapshots of the 64x32x32 torus, 32x32 camera
    "torus64_slow4_cam32": dict(grid=(64, 32, 32), n=32, spins=(0.9,), incs=(60.0,),
                                freqs=(230e9,), seed_index=5, snapshots=4, dt=10.0,
                                t_camera=1015.0),
}


def workload_inputs(name: str, spin: float, inc_deg: float, n: int | None = None):
    """Camera, metric and grid parameters plus the seeded torus (or snapshot series) for one
    image."""
    w = WORKLOADS[name]
    gp = grid_params_for(*w["grid"])
    cam = Camera(theta=math.radians(inc_deg), n=n if n is not None else w["n"])
    met = Metric(spin=spin)
    if w.get("snapshots", 1) > 1:
        gp = dataclasses.replace(gp, n_snapshots=w["snapshots"], time_interp=1, t_first=0.0,
                                 dt_snapshots=w["dt"], t_camera=w["t_camera"])
        prim = make_torus_series(gp, spin, BASE_SEED + w["seed_index"], w["snapshots"], w["dt"])
    else:
        prim = make_torus(gp, spin, BASE_SEED + w["seed_index"])
    return cam, met, gp, prim
