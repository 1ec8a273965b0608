"""The fixed-rule integrators (Sec. 2.2, Tables tab:rk2 and tab:rk4, Eq. rk_step) on the GPU
against the oracle: images, end states and step counts."""
import dataclasses

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


CAM, MET, GP, PRIM = S.workload_inputs("torus64_cam32", 0.9, 17.0)


def _rel_l2(got, want):
    nI = np.linalg.norm(want[:, 0])
    return [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]


@pytest.mark.parametrize("integrator", [native.BL_INT_RK4, native.BL_INT_RK2])
@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (1, 1e-3)])
def test_rk_image_and_end_states_vs_oracle(integrator, precision, tol):
    met = dataclasses.replace(MET, integrator=integrator, f_step=0.02)
    want = O.trace(CAM, met, GP, PRIM, 230e9)
    m = dataclasses.replace(met, precision=precision)
    p = torch.from_numpy(PRIM).to(DEV)
    rc, outs = images.trace_images([CAM], [m], [GP], [p], [230e9], end_state=True)
    torch.cuda.synchronize()
    o = outs[0]
    status = o["status"].cpu().numpy().reshape(-1)
    steps = o["steps"].cpu().numpy().reshape(-1)
    print("statuses gpu", np.unique(status, return_counts=True), "oracle",
          np.unique(want["status"], return_counts=True), "steps max", steps.max())
    assert rc == 0
    assert np.array_equal(status, want["status"])
    assert np.mean(steps == want["attempts"]) >= 0.99
    st = o["stokes"].double().cpu().numpy().reshape(4, -1).T
    err = _rel_l2(st, want["stokes"])
    print("rk", integrator, precision, "rel-L2", err)
    assert max(err) <= tol
    # final covariant momentum (independent of where the last step stops)
    end = o["end_state"].cpu().numpy().reshape(-1, 8)
    k, kw = end[:, 4:], want["end"][:, 4:]
    rel = np.max(np.abs(k - kw), axis=1) / np.max(np.abs(kw), axis=1)
    print("rk end momentum rel: median", np.median(rel), "max", rel.max())
    assert np.median(rel) <= 1e-12 and rel.max() <= 1e-8


def test_rk_arguments_are_checked():
    p = torch.from_numpy(PRIM).to(DEV)
    out = images.alloc_outputs(CAM.n, torch.float64)
    for bad in (dataclasses.replace(MET, integrator=1, f_step=0.0),
                dataclasses.replace(MET, integrator=1, f_step=1.5),
                dataclasses.replace(MET, integrator=7)):
        with pytest.raises(native.BlacklightError) as ei:
            native.blacklight_trace_batch([CAM], [bad], [GP], [p], [230e9], [out])
        assert ei.value.code == -1
    a = dataclasses.replace(MET, integrator=1, f_step=0.02)
    with pytest.raises(native.BlacklightError):
        native.blacklight_trace_batch([CAM, CAM], [a, MET], [GP, GP], [p, p], [230e9] * 2,
                                      [out, images.alloc_outputs(CAM.n, torch.float64)])
