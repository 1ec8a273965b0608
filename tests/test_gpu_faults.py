"""Defined outcomes for bad inputs and exhausted resources, all made on the host (no GPU fault):

  - grid cells holding NaN or infinite primitives: samples whose interpolation stencil touches
    them carry no plasma (vacuum there, as the oracle reads it), the trace returns 0 and no
    Stokes value is NaN;
  - a sample store that fills up (a tiny proper-length limit ds_max makes every step split
    into thousands of samples): the rays that do not fit end with status OVERFLOW (6) and
    NaN Stokes, the call returns BL_WRAYS, and the next trace on the same context is exact.
The termination rules and statuses follow the geodesics section."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.build()
    native.load()
    O.build()


def _rel_l2(got, want):
    nI = np.linalg.norm(want[:, 0])
    return [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]


def _poisoned_grid():
    gp = S.GridParams(n_r=64, n_theta=32, n_phi=32)
    prim = S.make_torus(gp, 0.9, S.BASE_SEED)
    clean = prim.copy()
    # blocks of cells inside the torus (r ~ 8-16 M near the midplane) in different fields
    prim[0, 0:6, 13:19, 30:34] = np.nan          # density
    prim[1, 10:14, 14:18, 26:30] = np.inf        # internal energy
    prim[5, 20:24, 12:20, 32:36] = -np.inf       # radial field
    prim[2, 26:30, 15:17, 28:31] = np.nan        # radial velocity
    return gp, prim, clean


@pytest.mark.parametrize("precision,tol", [(native.BL_PREC_FP64, 1e-6),
                                           (native.BL_PREC_FAST, 1e-3)])
def test_grid_with_nan_and_inf_cells(precision, tol):
    gp, prim, clean = _poisoned_grid()
    cam = S.Camera(theta=math.radians(60.0), n=24)
    met = S.Metric(spin=0.9, precision=precision)
    want = O.trace(cam, met, gp, prim, 230e9)
    want_clean = O.trace(cam, met, gp, clean, 230e9)
    # the poisoned cells are on the rays' paths: the image changes
    assert max(_rel_l2(want["stokes"], want_clean["stokes"])) > 1e-3
    assert np.all(np.isfinite(want["stokes"]))
    p = torch.from_numpy(prim).cuda()
    for layout in ("planes", "cells"):
        g, q = gp, p
        if layout == "cells":
            q, g = images.pack_grid(p, gp)
        rc, outs = images.trace_images([cam], [met], [g], [q], [230e9])
        torch.cuda.synchronize()
        assert rc == 0
        st = outs[0]["stokes"].double().cpu().numpy().reshape(4, -1).T
        assert np.all(np.isfinite(st))
        assert np.array_equal(outs[0]["status"].cpu().numpy().reshape(-1), want["status"])
        assert max(_rel_l2(st, want["stokes"])) <= tol


@pytest.mark.parametrize("precision", [native.BL_PREC_FP64, native.BL_PREC_FAST])
def test_sample_store_overflow(precision):
    gp = S.GridParams(n_r=64, n_theta=32, n_phi=32)
    prim = torch.from_numpy(S.make_torus(gp, 0.9, S.BASE_SEED)).cuda()
    cam = S.Camera(theta=math.radians(17.0), n=16)
    dt = torch.float64 if precision == native.BL_PREC_FP64 else torch.float32
    # every ray crosses the grid (r < 50 M inside the +-20 M field of view); at ds_max =
    # 1e-3 M a crossing needs ~1e5 samples against at most 4096 a ray
    bad = S.Metric(spin=0.9, precision=precision, ds_max=1e-3)
    out = images.alloc_outputs(cam.n, dt)
    rc = native.blacklight_trace(cam, bad, gp, prim, 230e9, out)
    torch.cuda.synchronize()
    assert rc == 1                      # BL_WRAYS
    status = out["status"].cpu().numpy()
    over = status == 6                  # BL_RAY_OVERFLOW
    assert over.mean() > 0.9
    st = out["stokes"].cpu().numpy()
    assert np.all(np.isnan(st[:, over]))
    # the context still works: a normal trace afterwards equals one in a fresh workspace
    good = S.Metric(spin=0.9, precision=precision)
    a = images.alloc_outputs(cam.n, dt)
    assert native.blacklight_trace(cam, good, gp, prim, 230e9, a) == 0
    b = images.alloc_outputs(cam.n, dt)
    assert native.blacklight_trace(cam, good, gp, prim, 230e9, b) == 0
    torch.cuda.synchronize()
    assert torch.equal(a["stokes"], b["stokes"]) and torch.equal(a["status"], b["status"])
    assert set(np.unique(a["status"].cpu().numpy())) <= {1, 2}
