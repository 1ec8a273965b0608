"""Learned coefficient model on the GPU against the oracle (oracle/mlp.py): training data,
the tensor-core forward pass and gradients (with the oracle rounding the same operands to
bfloat16), one Adam step, training, coefficients, and an image ablation."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as M
from paper_2203_15963_gb300 import coefmodel, images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.build()
    native.load()
    assert torch.cuda.is_available()


def _gpu(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(DEV)


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, M.N_PARAMS)
    p[M.OFF_MEAN:M.OFF_SCALE] = rng.normal(0.0, 1.0, 7)
    p[M.OFF_SCALE:M.OFF_A] = rng.uniform(0.5, 2.0, 7)
    p[M.OFF_A:] = rng.normal(0.0, 1.0, 21)
    return p.astype(np.float32).astype(np.float64)


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(*M.LX_RANGE, n), rng.uniform(*M.LT_RANGE, n),
                  rng.uniform(0, 1, n)], axis=1)
    return x.astype(np.float32).astype(np.float64)


def _features(x):
    """the oracle's network inputs at the float32 features the kernels compute"""
    f = M.features(x[:, 0], x[:, 1], x[:, 2])
    return f.astype(np.float32).astype(np.float64)


def test_dataset_is_uniform_and_targets_match_oracle():
    n = 4096
    inp = torch.empty((n, 3), dtype=torch.float32, device=DEV)
    tg = torch.empty((n, 7), dtype=torch.float32, device=DEV)
    native.blacklight_mlp_dataset(n, 12345, inp, tg)
    x = inp.double().cpu().numpy()
    assert x[:, 0].min() >= -3 and x[:, 0].max() <= 6 and abs(x[:, 0].mean() - 1.5) < 0.15
    assert x[:, 1].min() >= -1 and x[:, 1].max() <= 2 and abs(x[:, 1].mean() - 0.5) < 0.05
    assert x[:, 2].min() >= 0 and x[:, 2].max() <= 1
    sub = np.arange(0, n, 16)
    want = M.targets(x[sub, 0], x[sub, 1])
    got = tg.double().cpu().numpy()[sub]
    # float storage of O(10) values; Abramowitz-Stegun Bessel factors good to ~1e-7 relative
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5)
    # same inputs through the targets entry point: identical
    tg2 = torch.empty_like(tg)
    native.blacklight_mlp_targets(inp, tg2)
    assert torch.equal(tg, tg2)


def test_forward_matches_oracle_with_bf16_operands():
    p = _params(1)
    x = _inputs(1000, 2)                        # ragged: 7 full tiles and a partial one
    out = torch.empty((1000, 7), dtype=torch.float32, device=DEV)
    native.blacklight_mlp_forward(_gpu(p), _gpu(x), out)
    got = out.double().cpu().numpy()
    F = _features(x)
    want_q = M.outputs(p, F, quant=True)
    want = M.outputs(p, F, quant=False)
    sc = p[M.OFF_SCALE:M.OFF_A]
    dq = np.abs(got - want_q) / sc
    print("forward |gpu - oracle(bf16)| median", np.median(dq), "max", dq.max())
    assert np.median(dq) <= 1e-5
    assert dq.max() <= 5e-3          # an occasional operand rounded to the neighbouring bf16
    assert np.max(np.abs(got - want) / sc) <= 0.1


def _grad_abs(p, F, O, forward_roundings=6):
    """Magnitude bound of each gradient element's terms: the float64 backward pass of the same
    network with every operand replaced by its absolute value (|W|, |activations|, |SiLU'|),
    started from |E| plus the forward rounding error of the outputs, forward_roundings u
    (|H2| |W3|^T + |b3|) with u the bfloat16 unit roundoff."""
    d = M.unpack(p)
    n = F.shape[0]
    Y, c = M.forward(p, F, False)
    T = (np.asarray(O, dtype=np.float64) - M.trend(p, F)) / d["scale"]
    AY = np.abs(c["H2"]) @ np.abs(d["W3"]).T + np.abs(d["b3"])
    dY = 2.0 / (n * M.N_OUT) * (np.abs(Y - T) + forward_roundings * 2.0 ** -9 * AY)
    g = dict(W3=dY.T @ np.abs(c["H2"]), b3=dY.sum(axis=0))
    dZ2 = (dY @ np.abs(d["W3"])) * np.abs(M.silu_grad(c["Z2"]))
    g["W2"] = dZ2.T @ np.abs(c["H1"])
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ np.abs(d["W2"])) * np.abs(M.silu_grad(c["Z1"]))
    g["W1"] = dZ1.T @ np.abs(c["F"])
    g["mean"], g["scale"], g["A"] = np.zeros(M.N_OUT), np.zeros(M.N_OUT), np.zeros((M.N_OUT, 3))
    return M.pack(g)


def test_gradient_matches_oracle():
    """The tensor-core gradient element by element against the plain float64 backward pass.
    The kernels round every matrix-product operand to bfloat16 (unit roundoff u = 2^-9) and
    accumulate in FP32; a term of any gradient element passes through at most nine such
    roundings (inputs, W1, H1, W2, H2, W3, the output errors and the two back-propagated
    errors), so |g_gpu - g_64| <= 9 u g_abs, g_abs the same gradient with every operand
    replaced by its magnitude (cancellation between terms is what makes a relative bound per
    element impossible). FP32 accumulation adds ~n 2^-24 g_abs, negligible. The oracle with
    the same bf16 operand rounding is a secondary, tighter check."""
    p = _params(3)
    x = _inputs(424, 4)                         # 3 full tiles and a partial one
    rng = np.random.default_rng(5)
    o = (p[M.OFF_MEAN:M.OFF_SCALE] + p[M.OFF_SCALE:M.OFF_A] * rng.normal(0, 1, (424, 7)))
    o = o.astype(np.float32).astype(np.float64)
    g = torch.empty(M.N_PARAMS, dtype=torch.float32, device=DEV)
    loss = native.blacklight_mlp_grad(_gpu(p), _gpu(x), _gpu(o), g)
    got = g.double().cpu().numpy()
    F = _features(x)
    l64, want = M.loss_and_grad(p, F, o, quant=False)
    bound = 9 * 2.0 ** -9 * _grad_abs(p, F, o)
    tr = slice(0, M.OFF_MEAN)
    ratio = np.abs(got[tr] - want[tr]) / bound[tr]
    print("gradient |gpu - float64| / bound: max %.3f median %.3f" % (ratio.max(), np.median(ratio)))
    assert np.all(ratio <= 1.0), int(np.argmax(ratio))
    assert loss == pytest.approx(l64, rel=9 * 2.0 ** -9)
    # secondary: the oracle rounding the same operands to bfloat16 agrees to FP32 summation
    lq, want_q = M.loss_and_grad(p, F, o, quant=True)
    assert loss == pytest.approx(lq, rel=1e-4)
    blocks = {"W1": (M.OFF_W1, M.OFF_W2), "W2": (M.OFF_W2, M.OFF_B2), "b2": (M.OFF_B2, M.OFF_W3),
              "W3": (M.OFF_W3, M.OFF_B3), "b3": (M.OFF_B3, M.OFF_MEAN)}
    for name, (a, b) in blocks.items():
        eq = np.linalg.norm(got[a:b] - want_q[a:b]) / np.linalg.norm(want_q[a:b])
        assert eq <= 3e-3, name
    assert np.all(got[M.OFF_MEAN:] == 0.0)


def test_one_adam_step_matches_closed_form():
    """From zero moments the first Adam step moves each parameter by lr against the sign of
    its gradient (for |g| >> eps)."""
    p = _params(6)
    x = _inputs(256, 7)
    o = M.outputs(p, _features(x)) + 0.5
    pt = _gpu(p)
    g = torch.empty(M.N_PARAMS, dtype=torch.float32, device=DEV)
    native.blacklight_mlp_grad(pt, _gpu(x), _gpu(o), g)
    gg = g.double().cpu().numpy()
    hist = torch.zeros(1, dtype=torch.float32, device=DEV)
    native.blacklight_mlp_train(pt, _gpu(x), _gpu(o), 256, 1, 1e-3, 1e-3, loss_history=hist)
    p1 = pt.double().cpu().numpy()
    big = np.abs(gg[:M.OFF_MEAN]) > 1e-4 * np.abs(gg[:M.OFF_MEAN]).max()
    step = (p1 - p)[:M.OFF_MEAN]
    np.testing.assert_allclose(step[big], -1e-3 * np.sign(gg[:M.OFF_MEAN][big]), rtol=1e-3)
    assert np.all(p1[M.OFF_MEAN:] == p[M.OFF_MEAN:])
    assert float(hist[0]) == pytest.approx(M.loss_and_grad(p, _features(x), o, quant=True)[0],
                                           rel=1e-4)


@pytest.fixture(scope="module")
def trained():
    params, hist = coefmodel.train()
    torch.cuda.synchronize()
    return params, hist.cpu().numpy()


def test_training_converges(trained):
    params, hist = trained
    print("loss first/last", hist[0], hist[-200:].mean())
    assert hist[-200:].mean() < 1e-3 * hist[0]
    # held-out inputs: the model against the oracle's exact quantities (normalised error)
    x = _inputs(20000, 8)
    out = torch.empty((20000, 7), dtype=torch.float32, device=DEV)
    native.blacklight_mlp_forward(params, _gpu(x), out)
    want = M.targets(x[:, 0], x[:, 1])
    err = out.double().cpu().numpy() - want
    rms = np.sqrt(np.mean(err ** 2, axis=0))
    # o1-o3, o6, o7 are logarithms: an error e is a relative error e of the coefficient
    print("held-out rms error per output", rms)
    assert np.all(rms <= 4e-3)


def test_training_is_reproducible():
    """The tiles' gradient sums are reduced in a fixed order: two runs of the same recipe give
    the same parameters and loss history, bit for bit."""
    a, ha = coefmodel.train(seed=5, n=1 << 16, batch=4096, steps=300)
    b, hb = coefmodel.train(seed=5, n=1 << 16, batch=4096, steps=300)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(ha, hb)
    assert float(ha[-1]) < float(ha[0])


def _plasma(n, seed, in_domain=True):
    rng = np.random.default_rng(seed)
    rows = []
    while len(rows) < n:
        c = rng.uniform(-0.98, 0.98)
        th = 10.0 ** rng.uniform(-0.9, 1.9) if in_domain else 10.0 ** rng.uniform(-1.4, -1.05)
        b = 10.0 ** rng.uniform(-1, 2)
        nub = M._E * b / (2 * math.pi * M._ME * M._C)
        lx = rng.uniform(-2.5, 3.0)
        nu = 10.0 ** lx * 1.5 * nub * math.sqrt(1 - c * c) * th * th
        rows.append((10.0 ** rng.uniform(3, 6), th, b, nu, c))
    return np.array(rows)


def test_coefficients_with_model_and_exact_fallback(trained):
    params, _ = trained
    inp = _plasma(512, 9)
    out = torch.empty((512, 8), dtype=torch.float64, device=DEV)
    native.blacklight_mlp_coefficients(params, _gpu(inp, torch.float64), out)
    got = out.cpu().numpy()
    want = np.array([O.coefficients(*r) for r in inp])
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    # emission/absorption carry exp(o) factors: rms error of o ~ 1e-3 in natural-log units
    print("coefficient relative error, median per coefficient", np.median(rel, axis=0))
    assert np.all(np.median(rel[:, :6], axis=0) <= 1e-2)
    # outside the domain (Theta_e < 0.1): the FP32 exact fits (same device function)
    inp2 = _plasma(256, 10, in_domain=False)
    t2 = _gpu(inp2, torch.float64)
    a = torch.empty((256, 8), dtype=torch.float64, device=DEV)
    b = torch.empty((256, 8), dtype=torch.float64, device=DEV)
    native.blacklight_mlp_coefficients(params, t2, a)
    native.blacklight_coefficients(t2, b, native.BL_PREC_MIXED)
    torch.testing.assert_close(a, b, rtol=1e-6, atol=0.0)


def _rel_l2(got, want):
    nI = np.linalg.norm(want[:, 0])
    return [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]


def _image(cam, met, gp, prim, precision, coef_mlp=None):
    met = S.Metric(**{**met.__dict__, "precision": precision})
    rc, outs = images.trace_images([cam], [met], [gp], [_gpu(prim)], [230e9], coef_mlp=coef_mlp)
    torch.cuda.synchronize()
    assert rc == 0
    return outs[0]["stokes"].double().cpu().numpy().reshape(4, -1).T


def test_image_ablation_trained_model_vs_untrained_and_exact(trained):
    """Stokes image of the 32^2 parity case through the fused tensor-core transfer: the
    trained model against the oracle's exact coefficients, next to the same model before
    training and the exact FP32 path."""
    params, _ = trained
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 17.0)
    want = O.trace(cam, met, gp, prim, 230e9)["stokes"]
    exact = _rel_l2(_image(cam, met, gp, prim, native.BL_PREC_FAST), want)
    learned = _rel_l2(_image(cam, met, gp, prim, native.BL_PREC_FAST, params), want)
    init = torch.empty_like(params)
    native.blacklight_mlp_init(init, 20220330)
    init[M.OFF_MEAN:] = params[M.OFF_MEAN:]
    untrained = _rel_l2(_image(cam, met, gp, prim, native.BL_PREC_FAST, init), want)
    print("rel-L2 exact fits", exact, "trained model", learned, "untrained model", untrained)
    assert max(exact) <= 1e-5
    assert max(learned) <= 1e-3       # the image tolerance for the learned form
    assert max(learned) * 50 <= max(untrained)
