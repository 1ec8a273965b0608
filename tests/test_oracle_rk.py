"""Pins for the fixed-rule integrators of the oracle (Sec. 2.2, Tables tab:rk2 and tab:rk4,
Eq. rk_step): their order of accuracy on Kerr null geodesics, straight rays in flat space, and
the sample points."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2203_15963_gb300 import synth as S

CAM, MET, GP, PRIM = S.workload_inputs("torus64_cam32", 0.9, 60.0, n=8)


def _null_norm_drift(i, j, integrator, f_step):
    x, k, _, _, _ = O.camera_pixel(CAM, MET, i, j)
    m = dataclasses.replace(MET, integrator=integrator, f_step=f_step)
    r = O.geodesic(m, CAM.r, np.concatenate([x, k]))
    e = r["end"]
    _, ghi = O.metric_cks(e[:4], m.mass, m.spin)
    return r["status"], 0.5 * e[4:] @ ghi.reshape(4, 4) @ e[4:]


@pytest.mark.parametrize("integrator,order", [(1, 4), (2, 2)])
@pytest.mark.parametrize("pix", [(3, 5), (1, 6)])
def test_order_of_accuracy(integrator, order, pix):
    """The null condition H = g^ab k_a k_b / 2 = 0 drifts by the global truncation error:
    halving f_step divides the drift by 2^order (escaping rays, asymptotic regime)."""
    drifts = []
    for fs in (0.02, 0.01, 0.005):
        st, h = _null_norm_drift(*pix, integrator, fs)
        assert st == 2
        drifts.append(abs(h))
    want = 2.0 ** order
    for a, b in zip(drifts, drifts[1:]):
        assert 0.85 * want <= a / b <= 1.15 * want


@pytest.mark.parametrize("integrator", [1, 2])
def test_flat_space_rays_are_straight(integrator):
    m = dataclasses.replace(MET, flat=1, spin=0.0, integrator=integrator, f_step=0.05)
    x, k, _, _, _ = O.camera_pixel(CAM, m, 2, 3)
    r = O.geodesic(m, CAM.r, np.concatenate([x, k]), max_path=100000)
    assert r["status"] == 2
    path = r["path"][:, 1:4]
    d = path - x[1:4]
    # every point lies on the line through the start along the initial direction
    kdir = (path[-1] - x[1:4]) / np.linalg.norm(path[-1] - x[1:4])
    perp = d - np.outer(d @ kdir, kdir)
    assert np.max(np.linalg.norm(perp, axis=1)) <= 1e-9 * np.max(np.linalg.norm(d, axis=1))


def test_rk_samples_are_hermite_midpoints():
    """The sample of an unsubdivided step is (y0 + y1)/2 + h (f0 - f1)/8: on a straight flat
    ray it is the exact midpoint of the step."""
    m = dataclasses.replace(MET, flat=1, spin=0.0, integrator=1, f_step=0.05, ds_max=1e9)
    x, k, _, _, _ = O.camera_pixel(CAM, m, 2, 3)
    smp = O.ray_samples(m, GP, PRIM, CAM.r, np.concatenate([x, k]))
    xs, xn, dl = smp["x"], smp["node_x"], smp["dl"]
    # consecutive nodes bound each step; the sample sits halfway between them
    mid = 0.5 * (xn[:-1] + xn[1:])
    np.testing.assert_allclose(xs[:-1], mid, rtol=0, atol=1e-9 * CAM.r)


def _rk4_fine(y, h, m, n=16):
    """reference: n classical RK4 substeps of the geodesic equation written here from the
    right-hand side alone"""
    f = lambda v: O.geodesic_rhs(v, m.mass, m.spin)
    y = np.array(y, dtype=np.float64)
    d = h / n
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * d * k1)
        k3 = f(y + 0.5 * d * k2)
        k4 = f(y + d * k3)
        y = y + d * (k1 + 2 * k2 + 2 * k3 + k4) / 6.0
    return y


def test_rk_samples_match_the_state_half_a_step_on_in_curved_space():
    m = dataclasses.replace(MET, integrator=2, f_step=0.05, ds_max=1e9)
    x, k, _, _, _ = O.camera_pixel(CAM, m, 3, 5)
    smp = O.ray_samples(m, GP, PRIM, CAM.r, np.concatenate([x, k]))
    r_hor = 1.0 + np.sqrt(1.0 - m.spin ** 2)
    worst = 0.0
    for xs, ks, xn, kn, dl in zip(smp["x"], smp["k"], smp["node_x"], smp["node_k"], smp["dl"]):
        r0 = O.r_of_x(xn, m.spin)
        if r0 > 30.0:
            continue                      # near the hole, where the ray bends
        h = -m.f_step * (r0 - r_hor)
        assert dl == pytest.approx(abs(h), rel=1e-12)
        want = _rk4_fine(np.concatenate([xn, kn]), 0.5 * h, m)
        got = np.concatenate([xs, ks])
        worst = max(worst, np.max(np.abs(got - want)) / (abs(h) ** 2))
    # cubic Hermite: error O(h^4); the sign of the correction matters at O(h^2)
    assert 0.0 < worst < 1e-3
