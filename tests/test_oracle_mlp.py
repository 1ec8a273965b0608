"""Pins for the learned-coefficient oracle (oracle/mlp.py): the learned quantities against the
independently written full coefficient oracle and scipy's Bessel functions, the backward pass
against finite differences and a least-squares optimum, Adam's first step in closed form,
bfloat16 rounding on known values."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M


def test_bf16_rounding_known_values():
    got = M.bf16([1.0, 1.0 + 2.0 ** -8, 1.0 + 3.0 * 2.0 ** -8, math.pi, -2.5, 0.0, 1e-3])
    # ties go to the even mantissa: 1 + 2^-8 -> 1, 1 + 1.5 * 2^-7 -> 1 + 2^-6
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2.0 ** -6
    assert got[3] == 3.140625 and got[4] == -2.5 and got[5] == 0.0
    assert abs(got[6] - 1e-3) <= 1e-3 * 2.0 ** -8


def test_bessel_outputs_match_scipy():
    sp = pytest.importorskip("scipy.special")
    lt = np.array([-1.0, -0.5, 0.0, 0.7, 1.5, 2.0])
    o = M.targets(np.zeros_like(lt), lt)
    z = 1.0 / 10.0 ** lt
    np.testing.assert_allclose(o[:, 5], np.log(sp.kve(2, z)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(o[:, 6], np.log(sp.kv(0, z) / sp.kv(2, z)), rtol=0, atol=1e-11)


def _plasma_samples(n, seed):
    """Plasma states whose model inputs cover the trained domain."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        lx = rng.uniform(*M.LX_RANGE)
        lt = rng.uniform(*M.LT_RANGE)
        c = rng.uniform(-0.99, 0.99)
        b = 10.0 ** rng.uniform(-1, 2)
        th = 10.0 ** lt
        nub = M._E * b / (2 * math.pi * M._ME * M._C)
        nu = 10.0 ** lx * 1.5 * nub * math.sqrt(1 - c * c) * th * th
        out.append((10.0 ** rng.uniform(3, 7), th, b, nu, c))
    return out


def test_reconstruction_from_learned_quantities_equals_full_coefficients():
    """o1..o7 with the exact prefactors give the full coefficient oracle's eight values: pins
    the decomposition (a dropped factor or wrong power anywhere fails)."""
    for ne, th, b, nu, c in _plasma_samples(40, 1):
        lx, lt, ac = M.model_inputs(th, b, nu, c)
        assert M.in_domain(lx, lt)
        o = M.targets(np.array(lx), np.array(lt))
        got = M.reconstruct(o, ne, th, b, nu, c)
        want = O.coefficients(ne, th, b, nu, c)
        for k in range(8):
            assert got[k] == pytest.approx(want[k], rel=1e-9, abs=0.0), (k, got, want)


def _random_params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, M.N_PARAMS)
    p[M.OFF_MEAN:M.OFF_SCALE] = rng.normal(0.0, 1.0, 7)
    p[M.OFF_SCALE:M.OFF_A] = rng.uniform(0.5, 2.0, 7)
    p[M.OFF_A:] = rng.normal(0.0, 1.0, 21)
    return p


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    lx = rng.uniform(*M.LX_RANGE, n)
    lt = rng.uniform(*M.LT_RANGE, n)
    c = rng.uniform(0, 1, n)
    F = M.features(lx, lt, c)
    Ot = rng.normal(0.0, 1.0, (n, 7))
    return F, Ot


def test_backward_matches_central_differences():
    p = _random_params(2)
    F, Ot = _batch(33, 3)
    _, g = M.loss_and_grad(p, F, Ot)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(M.OFF_MEAN, 80, replace=False),
                          [M.OFF_W1 + 3, M.OFF_B2 + 5, M.OFF_B3 + 6]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, F, Ot)[0] - M.loss_and_grad(pm, F, Ot)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10), i
    assert np.all(g[M.OFF_MEAN:] == 0.0)


def test_zero_last_layer_blocks_gradient_to_earlier_layers():
    p = _random_params(5)
    p[M.OFF_W3:M.OFF_B3] = 0.0
    F, Ot = _batch(17, 6)
    d = M.unpack(p)
    np.testing.assert_allclose(M.outputs(p, F), d["mean"] + d["scale"] * d["b3"] + F[:, :3] @ d["A"].T,
                               rtol=1e-15, atol=1e-15)
    _, g = M.loss_and_grad(p, F, Ot)
    assert np.all(g[M.OFF_W1:M.OFF_W3] == 0.0)
    assert np.any(g[M.OFF_W3:M.OFF_B3] != 0.0) and np.all(g[M.OFF_B3:M.OFF_MEAN] != 0.0)


def test_least_squares_last_layer_has_zero_gradient():
    """With the hidden layers fixed, the output layer solving the linear least-squares problem
    is a stationary point of the loss: its W3 and b3 gradients vanish."""
    p = _random_params(7)
    F, Ot = _batch(200, 8)
    d = M.unpack(p)
    _, c = M.forward(p, F)
    T = (Ot - M.trend(p, F)) / d["scale"]
    A = np.hstack([c["H2"], np.ones((200, 1))])
    beta, *_ = np.linalg.lstsq(A, T, rcond=None)
    d["W3"] = beta[:64].T
    d["b3"] = beta[64]
    p2 = M.pack(d)
    _, g = M.loss_and_grad(p2, F, Ot)
    _, g0 = M.loss_and_grad(p, F, Ot)
    assert np.max(np.abs(g[M.OFF_W3:M.OFF_MEAN])) <= 1e-12 * np.max(np.abs(g0[M.OFF_W3:M.OFF_MEAN])) + 1e-15


def test_adam_first_step_is_a_signed_learning_rate():
    rng = np.random.default_rng(9)
    p = rng.normal(size=M.N_PARAMS)
    g = rng.normal(size=M.N_PARAMS)
    z = np.zeros(M.N_PARAMS)
    p1, m1, v1 = M.adam_step(p, g, z, z, 1, lr=1e-3)
    want = p[:M.OFF_MEAN] - 1e-3 * g[:M.OFF_MEAN] / (np.abs(g[:M.OFF_MEAN]) + 1e-8)
    np.testing.assert_allclose(p1[:M.OFF_MEAN], want, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(p1[M.OFF_MEAN:], p[M.OFF_MEAN:])


def test_quantized_forward_stays_within_bf16_rounding():
    p = _random_params(10, scale=0.2)
    F, _ = _batch(64, 11)
    y = M.forward(p, F)[0]
    yq = M.forward(p, F, quant=True)[0]
    # each product operand carries at most 2^-8 relative rounding; three layers deep
    assert np.max(np.abs(yq - y)) <= 0.05 * (np.max(np.abs(y)) + 1.0)
    assert np.max(np.abs(yq - y)) > 0.0


def test_affine_normalisation_reproduces_an_affine_target_exactly():
    """Targets that are affine in the inputs are taken up entirely by offset + A f (zero
    residual); a random non-affine remainder is orthogonal to (f, 1) afterwards."""
    F, _ = _batch(300, 12)
    rng = np.random.default_rng(13)
    A = rng.normal(size=(7, 3))
    c0 = rng.normal(size=7)
    O = c0 + F[:, :3] @ A.T
    d = M.affine_normalisation(F, O)
    np.testing.assert_allclose(d["A"], A, atol=1e-12)
    np.testing.assert_allclose(d["mean"], c0, atol=1e-12)
    assert np.all(d["scale"] < 1e-12)
    O2 = O + np.sin(5 * F[:, :1]) * np.ones((1, 7))
    d2 = M.affine_normalisation(F, O2)
    R = O2 - (d2["mean"] + F[:, :3] @ d2["A"].T)
    np.testing.assert_allclose(F.T @ R, 0.0, atol=1e-9)
    np.testing.assert_allclose(d2["scale"], np.sqrt(np.mean(R * R, axis=0)), rtol=1e-12)
