"""Pins for the oracle's adaptive-refinement criteria (Sec. 4) on fields with known
differences, and its level-0 reduction to the plain tracer."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import adaptive as A
from paper_2203_15963_gb300 import synth as S


def test_gradient_of_a_linear_ramp_is_its_slope():
    B = 6
    u = np.arange(B)
    I = 3.0 + 0.7 * u[None, :] - 0.2 * u[:, None]          # I[v][u]
    g = A.criterion_values(I, A.ABS_GRAD)
    assert np.allclose(g, math.hypot(0.7, 0.2), rtol=1e-14)
    assert np.allclose(A.criterion_values(I, A.ABS_LAPL), 0.0, atol=1e-13)


def test_laplacian_of_a_quadratic_and_relative_forms():
    B = 5
    u = np.arange(B, dtype=float)
    I = u[None, :] ** 2 + 2 * u[:, None] ** 2               # second differences 2 and 4
    assert np.allclose(A.criterion_values(I, A.ABS_LAPL), 6.0)
    k = 0.3
    E = np.exp(k * u)[None, :] * np.ones((B, 1))
    rel = A.criterion_values(E, A.REL_GRAD)
    # interior: 2 (e^k - e^-k) / (e^-k + 2 + e^k) = 2 tanh(k / 2)
    assert np.allclose(rel[:, 1:-1], 2 * math.tanh(k / 2), rtol=1e-13)
    # block edges, one-sided: 2 (e^k - 1) / (1 + e^k) = 2 tanh(k / 2) as well
    assert np.allclose(rel[:, [0, -1]], 2 * math.tanh(k / 2), rtol=1e-13)
    rl = A.criterion_values(E, A.REL_LAPL)
    # 4 (e^-k - 2 + e^k) / (e^-k + 2 + e^k) = 4 tanh^2(k / 2)
    assert np.allclose(rl, 4 * math.tanh(k / 2) ** 2, rtol=1e-12)


def test_refinement_count_and_dark_blocks():
    I = np.zeros((4, 4))
    assert not A.refines(I, A.REL_GRAD, 0.1, 1)             # 0/0 never counts
    I[1, 1] = 1.0
    vals = A.criterion_values(I, A.ABS_GRAD)
    assert A.refines(I, A.ABS_GRAD, 0.4, int(np.sum(vals > 0.4)))
    assert not A.refines(I, A.ABS_GRAD, 0.4, int(np.sum(vals > 0.4)) + 1)
    assert not A.refines(np.full((8, 8), 2.5), A.ABS_GRAD, 0.0, 1)


def test_level_zero_is_the_plain_image():
    gp = S.GridParams(n_r=32, n_theta=16, n_phi=16)
    prim = S.make_torus(gp, 0.5, seed=3)
    cam = S.Camera(theta=math.radians(40), n=8)
    met = S.Metric(spin=0.5)
    comp, lr = A.trace_adaptive(cam, met, gp, prim, 230e9, 4, 0, A.REL_GRAD, 0.1, 5)
    plain = O.trace(cam, met, gp, prim, 230e9)["stokes"].T.reshape(4, 8, 8)
    assert np.array_equal(comp, plain) and list(lr) == [64]
