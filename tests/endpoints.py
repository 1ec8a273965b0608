"""Comparison of geodesic end states (test helper).

A traced ray stops after the accepted step whose end lies beyond the camera sphere r = r_cam
(the escape rule of the geodesics section), so two integrations of the same ray whose step
sequences differ stop at different points on it. Two ways of comparing them:

  - `cut_free_error`: for rays with the same step sequence, the quantities that do not
    depend on where the ray was cut -- the final momentum, the position transverse to it and
    the axial angular momentum L_z = x k_y - y k_x (a constant of the motion in Kerr-Schild
    coordinates, which are axisymmetric about z);
  - `at_camera_sphere`: any end state carried back along its geodesic to r = r_cam with the
    oracle's right-hand side (fine fixed-step RK4 near r_cam, where the ray is nearly
    straight), after which full states can be compared.
"""
import numpy as np

import oracle as O


def cut_free_error(ge, oe):
    """Largest relative difference, per ray, of momentum, transverse position and L_z
    between end states ge and oe ([n][8]: t, x, y, z, k_t, k_x, k_y, k_z)."""
    kg, ko = ge[:, 5:8], oe[:, 5:8]
    kn = np.linalg.norm(ko, axis=1)
    khat = ko / kn[:, None]

    def perp(x):
        return x - np.sum(x * khat, axis=1)[:, None] * khat

    ek = np.linalg.norm(kg - ko, axis=1) / kn
    ex = (np.linalg.norm(perp(ge[:, 1:4]) - perp(oe[:, 1:4]), axis=1) /
          np.linalg.norm(oe[:, 1:4], axis=1))
    lz_g = ge[:, 1] * ge[:, 6] - ge[:, 2] * ge[:, 5]
    lz_o = oe[:, 1] * oe[:, 6] - oe[:, 2] * oe[:, 5]
    el = np.abs(lz_g - lz_o) / (np.abs(lz_o) + 1.0)
    return np.maximum(np.maximum(ek, ex), el)


def _rk4(y, h, mass, spin):
    k1 = O.geodesic_rhs(y, mass, spin)
    k2 = O.geodesic_rhs(y + 0.5 * h * k1, mass, spin)
    k3 = O.geodesic_rhs(y + 0.5 * h * k2, mass, spin)
    k4 = O.geodesic_rhs(y + h * k3, mass, spin)
    return y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)


def at_camera_sphere(y, mass, spin, r_cam, max_sub=2.0):
    """The state on the same geodesic where r = r_cam: Newton iterations on r(lambda), each
    an RK4 integration (substeps of at most max_sub in affine parameter) by
    (r_cam - r) / (dr/dlambda)."""
    y = np.array(y, dtype=np.float64)
    for _ in range(20):
        r = O.r_of_x(y[:4], spin)
        if abs(r - r_cam) <= 1e-13 * r_cam:
            break
        f = O.geodesic_rhs(y, mass, spin)
        eps = 1e-3
        drdl = (O.r_of_x(y[:4] + eps * f[:4], spin) - O.r_of_x(y[:4] - eps * f[:4], spin)) / (2 * eps)
        dl = (r_cam - r) / drdl
        n = max(1, int(np.ceil(abs(dl) / max_sub)))
        for _ in range(n):
            y = _rk4(y, dl / n, mass, spin)
    return y


def camera_sphere_error(ga, ob, mass, spin, r_cam):
    """Relative difference of position and momentum of two end states of one ray after both
    are carried to r = r_cam."""
    a = at_camera_sphere(ga, mass, spin, r_cam)
    b = at_camera_sphere(ob, mass, spin, r_cam)
    ex = np.linalg.norm(a[1:4] - b[1:4]) / np.linalg.norm(b[1:4])
    ek = np.linalg.norm(a[5:8] - b[5:8]) / np.linalg.norm(b[5:8])
    return max(ex, ek)
