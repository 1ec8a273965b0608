"""Stencil field test (Secs. 2.4-2.5): a sample whose lookup stencil holds no magnetic field has
b = 0 and no synchrotron plasma, so the library skips its interpolation and plasma state (the
FP64 sample pass decides it in FP32 from the record's position with a margin on every axis).
The skip must be exact. Here the torus keeps its field only in alternating 2x2x2 blocks of
cells (shifted from snapshot to snapshot in a slow-light series), so that a large share of the
samples lie on stencils that straddle a field / no-field boundary: the FP64 image must still
match the oracle to the full-size bound (a wrongly skipped emitting sample moves a pixel by far
more), and the FP32 transfer with the test (plane-layout grid, consecutive queue) must equal
the one without it (cell layout, record-count queue) bit for bit."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"
FREQ = 230e9


def _blocky(workload, spin, inc):
    """The workload's torus with its field kept only in alternating 2x2x2 blocks of cells (in a
    snapshot series, the blocks shift by one block from snapshot to snapshot)."""
    cam, met, gp, prim = S.workload_inputs(workload, spin, inc, n=48)
    prim = np.array(prim, copy=True)
    k, j, i = np.meshgrid(np.arange(gp.n_phi), np.arange(gp.n_theta), np.arange(gp.n_r),
                          indexing="ij")
    snaps = prim if prim.ndim == 5 else prim[None]
    for s_ in range(snaps.shape[0]):
        keep = ((i // 2 + j // 2 + k // 2 + s_) % 2 == 0).astype(np.float32)
        for v in (5, 6, 7):
            snaps[s_, v] *= keep
    return cam, met, gp, prim


@pytest.fixture(scope="module")
def blocky():
    native.build()
    native.load()
    O.build()
    return _blocky("torus64_cam32", 0.9, 60.0)


def _trace(cam, met, gp, prim_dev, dtype):
    out = images.alloc_outputs(cam.n, dtype, device=DEV)
    rc = native.blacklight_trace_batch([cam], [met], [gp], [prim_dev], [FREQ], [out])
    torch.cuda.synchronize()
    assert rc == 0
    return out


@pytest.mark.parametrize("layout,interp,slow", [("planes", 1, False), ("cells", 1, False),
                                                 ("cells", 0, False), ("cells", 1, True),
                                                 ("planes", 0, True)])
def test_fp64_image_with_blocky_field_matches_oracle(blocky, layout, interp, slow):
    """Trilinear and nearest lookup, one snapshot and a slow-light series (the stencil must be
    field-free in both snapshots a sample interpolates between)."""
    cam, met, gp, prim = _blocky("torus64_slow4_cam32", 0.9, 60.0) if slow else blocky
    gp = dataclasses.replace(gp, interp=interp)
    met = dataclasses.replace(met, precision=native.BL_PREC_FP64)
    p = torch.from_numpy(prim).to(DEV)
    g = gp
    if layout == "cells":
        p, g = images.pack_grid(p, gp)
    out = _trace(cam, met, g, p, torch.float64)
    ora = O.trace(cam, met, gp, prim, FREQ)
    got = out["stokes"].cpu().numpy().reshape(4, -1).T
    want = ora["stokes"]
    assert np.sum(want[:, 0]) > 0.0
    nI = np.linalg.norm(want[:, 0])
    err = [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]
    print("rel-L2", err)
    assert max(err) <= 1e-7, err
    assert np.array_equal(out["status"].cpu().numpy().reshape(-1), ora["status"])


@pytest.mark.parametrize("precision", [native.BL_PREC_FAST, native.BL_PREC_MIXED])
def test_fp32_field_test_changes_no_bit(blocky, precision):
    cam, met, gp, prim = blocky
    met = dataclasses.replace(met, precision=precision)
    planes = torch.from_numpy(prim).to(DEV)
    cells, gpc = images.pack_grid(planes, gp)
    with_test = _trace(cam, met, gp, planes, torch.float32)
    without = _trace(cam, met, gpc, cells, torch.float32)
    assert float(with_test["stokes"].abs().sum()) > 0.0
    for k in with_test:
        assert torch.equal(with_test[k], without[k]), k
