"""Pins for slow light in the oracle (Sec. 4, "Slow Light"): fluid data interpolated in time
along the ray. A field linear in time is reproduced exactly between snapshots (and clamped
outside them, and rounded to the nearest snapshot in nearest mode); identical snapshots give
the fast-light image; the samples' coordinate times follow the light travel time."""
import ctypes
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2203_15963_gb300 import synth as S


def _const_series(gp, n, base, slope, t_first, dt):
    """snapshots whose every cell holds base[v] + slope[v] t_s"""
    shape = (8, gp.n_phi, gp.n_theta, gp.n_r)
    out = np.empty((n,) + shape, dtype=np.float32)
    for s in range(n):
        t = t_first + s * dt
        for v in range(8):
            out[s, v] = base[v] + slope[v] * t
    return out


def _point(r, th, ph):
    return np.array([0.0, r * math.sin(th) * math.cos(ph), r * math.sin(th) * math.sin(ph),
                     r * math.cos(th)])


@pytest.mark.parametrize("interp", [1, 0])
def test_linear_in_time_field_is_reproduced(interp):
    gp0 = S.GridParams(n_r=8, n_theta=4, n_phi=4)
    gp = dataclasses.replace(gp0, n_snapshots=5, time_interp=interp, t_first=100.0,
                             dt_snapshots=10.0, t_camera=1000.0)
    base = np.arange(1, 9, dtype=np.float64)
    slope = np.array([0.5, -0.25, 0.125, 0.0, 1.0, -1.0, 0.0625, 2.0])
    prim = _const_series(gp, 5, base, slope, gp.t_first, gp.dt_snapshots)
    for xt in (-900.0, -887.5, -871.25, -850.0, -1000.0, -700.0):
        x = _point(10.0, 1.1, 0.7)
        x[0] = xt
        gs = O.grid_struct(gp, prim)
        got = np.zeros(8)
        ok = O.lib().ora_sample_grid(ctypes.byref(gs), 0.0, O._p(np.ascontiguousarray(x)),
                                     O._p(got))
        assert ok == 1
        t = min(max(gp.t_camera + xt, 100.0), 140.0)       # clamped to the snapshot span
        if interp == 0:
            t = 100.0 + 10.0 * math.floor((t - 100.0) / 10.0 + 0.5)
        np.testing.assert_allclose(got, base + slope * t, rtol=1e-6, atol=1e-6)


def test_identical_snapshots_give_the_fast_light_image():
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 17.0, n=12)
    fast = O.trace(cam, met, gp, prim, 230e9)
    gps = dataclasses.replace(gp, n_snapshots=3, time_interp=1, t_first=0.0, dt_snapshots=7.0,
                              t_camera=1003.0)
    series = np.ascontiguousarray(np.stack([prim, prim, prim]))
    slow = O.trace(cam, met, gps, series, 230e9)
    np.testing.assert_array_equal(slow["status"], fast["status"])
    np.testing.assert_allclose(slow["stokes"], fast["stokes"], rtol=1e-12, atol=0.0)


def test_sample_times_follow_the_light_travel_time():
    """Rays are traced backward from the camera at t = 0: a sample at radius r left the
    plasma about r_cam - r earlier (the Kerr-Schild time delay adds 2 ln terms of order 10 M)."""
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 17.0, n=8)
    x, k, _, _, _ = O.camera_pixel(cam, met, 4, 4)
    smp = O.ray_samples(met, gp, prim, cam.r, np.concatenate([x, k]))
    assert len(smp["dl"]) > 10
    for xs in smp["x"]:
        r = O.r_of_x(xs, met.spin)
        delay = -xs[0] - (cam.r - r)
        assert 0.0 <= delay <= 60.0, (r, xs[0])
