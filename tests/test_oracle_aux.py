"""Pins for the unpolarized transfer (Eq. unpolarized) and the auxiliary images (Sec. 4,
"Auxiliary Images") of the oracle."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2203_15963_gb300 import synth as S


@pytest.mark.parametrize("j,alpha,dl,i0", [(2.0, 0.5, 3.0, 0.7), (1e-3, 2.0, 0.1, 5.0),
                                           (4.0, 0.0, 2.5, 1.0), (3.0, 80.0, 2.0, 9.0)])
def test_unpolarized_step_cases_and_agreement_with_the_stokes_step(j, alpha, dl, i0):
    got = O.unpolarized_step(j, alpha, dl, i0)
    if alpha == 0.0:
        want = i0 + j * dl
    elif alpha * dl >= 100.0:
        want = j / alpha
    else:
        want = (j / alpha) + (i0 - j / alpha) * math.exp(-alpha * dl)   # uniform slab
    assert got == pytest.approx(want, rel=1e-14, abs=0.0)
    # the polarized step (matrix exponential) with only the I coefficients reduces to it
    if alpha * dl < 100.0:
        s1 = O.stokes_step([j, 0, 0, alpha, 0, 0, 0, 0], [i0, 0, 0, 0], dl)
        assert s1[0] == pytest.approx(got, rel=1e-13, abs=0.0)
    # two half segments compose to the whole segment
    half = O.unpolarized_step(j, alpha, dl / 2, O.unpolarized_step(j, alpha, dl / 2, i0))
    if alpha * dl < 100.0:
        assert half == pytest.approx(got, rel=1e-13, abs=0.0)


def test_flat_spacetime_time_equals_length():
    """In flat spacetime seen by the static camera light moves at unit speed: the elapsed time
    equals the proper length, and the affine parameter is that length over |k^t|."""
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.0, 60.0, n=6)
    met = dataclasses.replace(met, flat=1)
    res = O.trace(cam, met, gp, prim, 230e9, aux=True)
    aux = res["aux"]
    assert np.all(aux[:, 0] > 900.0)
    np.testing.assert_allclose(aux[:, 1], aux[:, 0], rtol=1e-9)
    kt = np.abs(res["end"][:, 4])
    np.testing.assert_allclose(aux[:, 2] * kt, aux[:, 1], rtol=1e-9)


def _uniform_grid(gp):
    """constant primitives: rho, u_gas, static fluid, a weak field along theta"""
    prim = np.zeros((8, gp.n_phi, gp.n_theta, gp.n_r), dtype=np.float32)
    prim[0] = 0.5
    prim[1] = 0.05
    prim[6] = 1e-3
    return prim


def test_uniform_plasma_averages_have_closed_forms():
    cam, met, gp, _ = S.workload_inputs("torus64_cam32", 0.5, 60.0, n=6)
    gp = dataclasses.replace(gp, r_high=1.0, r_low=1.0)      # T_i = T_e: Theta_e uniform
    prim = _uniform_grid(gp)
    res = O.trace(cam, met, gp, prim, 230e9, aux=True)
    aux = res["aux"]
    ok, pl = O.plasma(gp, prim, met, np.array([0.0, 10.0, 0.0, 3.0]))
    assert ok
    rho, ne, theta = 0.5, pl["ne"], pl["theta_e"]
    p = (gp.gamma_ad - 1.0) * float(np.float32(0.05))
    tau = aux[:, 4]
    assert np.all(aux[:, 3] > 0.0) and np.all(tau > 0.0)
    for k, q in ((0, rho), (1, ne), (2, p), (3, theta)):
        np.testing.assert_allclose(aux[:, 12 + k], q, rtol=1e-6)                   # <q>_Ij
        np.testing.assert_allclose(aux[:, 19 + k], q * -np.expm1(-tau), rtol=1e-9)  # <q>_tau
        assert np.all(aux[:, 5 + k] > 0.0) and np.all(aux[:, 5 + k] < q)           # <q>_lambda


def test_unpolarized_intensity_lies_between_attenuated_and_total_emission():
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 17.0, n=8)
    res = O.trace(cam, met, gp, prim, 230e9, unpolarized=True, aux=True)
    I = res["stokes"][:, 0]
    Ij, tau = res["aux"][:, 3], res["aux"][:, 4]
    assert np.all(res["stokes"][:, 1:] == 0.0)
    assert np.all(I <= Ij * (1 + 1e-12))
    assert np.all(I >= Ij * np.exp(-tau) * (1 - 1e-12))
    assert np.any(tau > 1e-3)
    # the polarized image's I is close to the unpolarized one for this weakly polarized source
    pol = O.trace(cam, met, gp, prim, 230e9)["stokes"][:, 0]
    assert np.linalg.norm(pol - I) / np.linalg.norm(I) < 0.2
