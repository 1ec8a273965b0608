"""Slow light (Sec. 4, "Slow Light") on the GPU against the oracle: fluid data interpolated in
time along each ray from a series of snapshots of the rotating torus."""
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


SLOW = S.workload_inputs("torus64_slow4_cam32", 0.9, 60.0)


def _rel_l2(got, want):
    nI = np.linalg.norm(want[:, 0])
    return [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]


def _gpu_image(cam, met, gp, prim, precision):
    met = S.Metric(**{**met.__dict__, "precision": precision})
    p = torch.from_numpy(np.ascontiguousarray(prim)).to(DEV)
    rc, outs = images.trace_images([cam], [met], [gp], [p], [230e9])
    torch.cuda.synchronize()
    o = outs[0]
    return rc, o["stokes"].double().cpu().numpy().reshape(4, -1).T, o["status"].cpu().numpy().reshape(-1)


@pytest.fixture(scope="module")
def slow_oracle():
    cam, met, gp, prim = SLOW
    return O.trace(cam, met, gp, prim, 230e9)


@pytest.mark.parametrize("precision,tol", [(native.BL_PREC_FP64, 1e-6), (native.BL_PREC_FAST, 1e-3)])
def test_slow_light_image_vs_oracle(slow_oracle, precision, tol):
    cam, met, gp, prim = SLOW
    rc, st, status = _gpu_image(cam, met, gp, prim, precision)
    assert rc == 0
    assert np.array_equal(status, slow_oracle["status"])
    err = _rel_l2(st, slow_oracle["stokes"])
    print("slow light rel-L2", precision, err)
    assert max(err) <= tol


def test_nearest_snapshot_mode_vs_oracle():
    cam, met, gp, prim = SLOW
    gp = dataclasses.replace(gp, time_interp=0)
    want = O.trace(cam, met, gp, prim, 230e9)
    rc, st, status = _gpu_image(cam, met, gp, prim, native.BL_PREC_FP64)
    assert rc == 0 and np.array_equal(status, want["status"])
    assert max(_rel_l2(st, want["stokes"])) <= 1e-6


def test_identical_snapshots_reproduce_fast_light_and_slow_light_differs():
    cam, met, gp, prim = SLOW
    gp1 = dataclasses.replace(gp, n_snapshots=1)
    one = np.ascontiguousarray(prim[1])
    _, fast, _ = _gpu_image(cam, met, gp1, one, native.BL_PREC_FP64)
    same = np.ascontiguousarray(np.stack([one] * 4))
    _, slow_same, _ = _gpu_image(cam, met, gp, same, native.BL_PREC_FP64)
    assert max(_rel_l2(slow_same, fast)) <= 1e-12
    _, slow, _ = _gpu_image(cam, met, gp, prim, native.BL_PREC_FP64)
    assert max(_rel_l2(slow, fast)) > 1e-3        # the rotating series changes the image


def test_slow_light_plan_and_invalid_arguments():
    cam, met, gp, prim = SLOW
    met = S.Metric(**{**met.__dict__, "precision": native.BL_PREC_FAST})
    p = torch.from_numpy(np.ascontiguousarray(prim)).to(DEV)
    ref = [images.alloc_outputs(cam.n, torch.float32, device=DEV)]
    native.blacklight_trace_batch([cam], [met], [gp], [p], [230e9], ref)
    outs = [images.alloc_outputs(cam.n, torch.float32, device=DEV)]
    plan = native.Plan([cam], [met], [gp], [p], [230e9], outs)
    plan.run()
    plan.check()
    assert torch.equal(outs[0]["stokes"], ref[0]["stokes"])
    plan.close()
    for bad in (dataclasses.replace(gp, dt_snapshots=0.0), dataclasses.replace(gp, time_interp=3)):
        with pytest.raises(native.BlacklightError) as ei:
            native.blacklight_trace_batch([cam], [met], [bad], [p], [230e9], ref)
        assert ei.value.code == -1
