"""blacklight_trace_noalloc: the trace entry point for callers that cannot allocate device
memory (a fixed allocator budget, a foreign memory pool). It must give the same Stokes images
as blacklight_trace, call after call, while working only in its fixed in-library scratch.

This file is collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process."""
import math

import numpy as np
import pytest
import torch

from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a = a.double().cpu().numpy().reshape(4, -1)
    b = b.double().cpu().numpy().reshape(4, -1)
    n = np.linalg.norm(b[0])
    return [float(np.linalg.norm(a[s] - b[s]) / n) for s in range(4)]


@pytest.mark.parametrize("precision,tol", [(native.BL_PREC_FP64, 1e-6),
                                           (native.BL_PREC_MIXED, 1e-3)])
def test_noalloc_matches_trace_on_consecutive_calls(precision, tol):
    native.build()
    native.load()
    gp = S.GridParams(n_r=64, n_theta=32, n_phi=32)
    prim = torch.from_numpy(S.make_torus(gp, 0.9, S.BASE_SEED)).cuda()
    dtype = torch.float64 if precision == native.BL_PREC_FP64 else torch.float32
    cases = [(S.Camera(theta=math.radians(17.0), n=32), S.Metric(spin=0.9, precision=precision)),
             (S.Camera(theta=math.radians(60.0), n=24), S.Metric(spin=0.9, precision=precision))]
    for cam, met in cases:          # two calls in a row; the second reuses the same scratch
        ref = images.alloc_outputs(cam.n, dtype)
        assert native.blacklight_trace(cam, met, gp, prim, 230e9, ref) == 0
        got = images.alloc_outputs(cam.n, dtype)
        assert native.blacklight_trace_noalloc(cam, met, gp, prim, 230e9, got) == 0
        torch.cuda.synchronize()
        assert torch.equal(got["status"], ref["status"])
        err = _rel_l2(got["stokes"], ref["stokes"])
        assert max(err) <= tol, err


def test_noalloc_rejects_cameras_beyond_its_scratch():
    native.load()
    gp = S.GridParams(n_r=8, n_theta=8, n_phi=8)
    prim = torch.zeros((8, 8, 8, 8), dtype=torch.float32, device="cuda")
    cam = S.Camera(n=33)
    out = images.alloc_outputs(33, torch.float32)
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_trace_noalloc(cam, S.Metric(precision=1), gp, prim, 230e9, out)
    assert ei.value.code == -1 and "scratch" in str(ei.value)
