"""Unpolarized transfer (Eq. unpolarized) and the auxiliary images (Sec. 4, "Auxiliary
Images") on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.build()
    native.load()
    assert torch.cuda.is_available()


C1 = S.workload_inputs("torus64_cam32", 0.9, 17.0)


def _rel_l2(got, want):
    nI = np.linalg.norm(want[:, 0])
    return [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]


def _gpu(cam, met, gp, prim, precision, flags=0, aux=False):
    met = S.Metric(**{**met.__dict__, "precision": precision})
    p = torch.from_numpy(prim).to(DEV)
    rc, outs = images.trace_images([cam], [met], [gp], [p], [230e9], flags=flags, aux=aux)
    torch.cuda.synchronize()
    o = outs[0]
    res = dict(rc=rc, stokes=o["stokes"].double().cpu().numpy().reshape(4, -1).T,
               status=o["status"].cpu().numpy().reshape(-1))
    if aux:
        res["aux"] = o["aux"].double().cpu().numpy().reshape(26, -1).T
    return res


@pytest.fixture(scope="module")
def oracle_unpol():
    cam, met, gp, prim = C1
    return O.trace(cam, met, gp, prim, 230e9, unpolarized=True, aux=True)


@pytest.fixture(scope="module")
def oracle_pol():
    cam, met, gp, prim = C1
    return O.trace(cam, met, gp, prim, 230e9, aux=True)


@pytest.mark.parametrize("precision,tol", [(native.BL_PREC_FP64, 1e-6), (native.BL_PREC_FAST, 1e-3)])
def test_unpolarized_image_vs_oracle(oracle_unpol, precision, tol):
    cam, met, gp, prim = C1
    g = _gpu(cam, met, gp, prim, precision, flags=native.BL_UNPOLARIZED)
    assert g["rc"] == 0 and np.array_equal(g["status"], oracle_unpol["status"])
    assert np.all(g["stokes"][:, 1:] == 0.0)
    err = _rel_l2(g["stokes"], oracle_unpol["stokes"])[0]
    print("unpolarized rel-L2", precision, err)
    assert err <= tol


def _aux_errors(got, want):
    """per-plane error: geodesic planes relative per pixel (median, max); integral and average
    planes as relative L2 over the image, the emission-weighted averages over the pixels whose
    I_j is at least 1e-6 of the image's largest (elsewhere the average has no weight: in FP32
    the emissivities of numerically dark rays flush to zero)"""
    out = {}
    bright = want[:, 3] >= 1e-6 * want[:, 3].max()
    for a in range(26):
        g, w = got[:, a], want[:, a]
        if a < 3:
            rel = np.abs(g - w) / np.abs(w)
            out[a] = (float(np.median(rel)), float(np.max(rel)))
            continue
        if 12 <= a <= 18:
            g, w = g[bright], w[bright]
        nw = np.linalg.norm(w)
        out[a] = float(np.linalg.norm(g - w) / nw) if nw > 0 else float(np.linalg.norm(g))
    return out


@pytest.mark.parametrize("precision,tol", [(native.BL_PREC_FP64, 1e-6), (native.BL_PREC_FAST, 2e-3)])
def test_aux_images_vs_oracle(oracle_pol, precision, tol):
    cam, met, gp, prim = C1
    g = _gpu(cam, met, gp, prim, precision, aux=True)
    assert g["rc"] == 0
    err = _aux_errors(g["aux"], oracle_pol["aux"])
    print("aux errors", precision, err)
    # time, length and affine parameter depend on where the integration stops, which rounding
    # in the step-size control moves by parts in 1e9 (FP64) to 1e6 (FP32 step control)
    for a in range(3):
        med, mx = err[a]
        fp64 = precision == native.BL_PREC_FP64
        assert med <= (1e-8 if fp64 else 5e-6)
        assert mx <= (1e-6 if fp64 else 5e-5)
    for a in range(3, 26):
        assert err[a] <= tol, a
    # asking for auxiliary images leaves the Stokes image unchanged up to rounding (another
    # compiled variant of the transfer kernel)
    g0 = _gpu(cam, met, gp, prim, precision)
    assert max(_rel_l2(g["stokes"], g0["stokes"])) <= (1e-12 if precision == 0 else 1e-6)


def test_unpolarized_with_aux_and_learned_model_rejected(oracle_unpol):
    cam, met, gp, prim = C1
    g = _gpu(cam, met, gp, prim, native.BL_PREC_FP64, flags=native.BL_UNPOLARIZED, aux=True)
    err = _aux_errors(g["aux"], oracle_unpol["aux"])
    assert max(err[a] for a in range(3, 26)) <= 1e-6
    met2 = S.Metric(**{**met.__dict__, "precision": native.BL_PREC_FAST})
    p = torch.from_numpy(prim).to(DEV)
    params = torch.zeros(native.MLP_PARAMS, dtype=torch.float32, device=DEV)
    out = images.alloc_outputs(cam.n, torch.float32)
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_trace_batch([cam], [met2], [gp], [p], [230e9], [out],
                                      flags=native.BL_UNPOLARIZED, coef_mlp=params)
    assert ei.value.code == -4
