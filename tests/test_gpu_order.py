"""Work-ordered ray queue. The DP integrator (Sec. 2.2, Table tab:dp) takes a varying number
of attempts per ray, so the library queues a large enough batch as 8x8 pixel blocks, longest
predicted work first (the prediction: each block's centre ray integrated beforehand). The
order is scheduling only: every ray is computed the same way in any queue order, so a
work-ordered trace equals the Morton-ordered plan bit for bit, in every precision form, in
one wave or several, and the geodesic-only path agrees with the traced end states."""
import pytest
import torch

from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"
FREQ = 230e9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.build()
    native.load()
    assert torch.cuda.is_available()


def _batch(precision, n=128, cells=True):
    """Four 128x128 images (65536 rays: the smallest batch the queue is reordered for), grids
    in the cell layout (the plane layout keeps the consecutive queue)."""
    cams, mets, gps, prims = [], [], [], []
    for spin, inc in ((0.94, 17.0), (0.5, 60.0), (0.0, 90.0), (0.94, 60.0)):
        cam, met, gp, prim = S.workload_inputs("torus64_cam32", spin, inc, n=n)
        p = torch.from_numpy(prim).to(DEV)
        if cells:
            p, gp = images.pack_grid(p, gp)
        cams.append(cam)
        mets.append(S.Metric(**{**met.__dict__, "precision": precision}))
        gps.append(gp)
        prims.append(p)
    return cams, mets, gps, prims


def _dtype(precision):
    return torch.float64 if precision == native.BL_PREC_FP64 else torch.float32


def _outs(cams, dtype, end_state=False):
    return [images.alloc_outputs(c.n, dtype, device=DEV, samples=True, end_state=end_state)
            for c in cams]


def _same(a, b, keys=("stokes", "status", "steps", "samples")):
    for x, y in zip(a, b):
        for k in keys:
            assert torch.equal(x[k], y[k]), k


@pytest.mark.parametrize("precision", [native.BL_PREC_FAST, native.BL_PREC_MIXED,
                                       native.BL_PREC_FP64])
def test_work_ordered_trace_equals_morton_plan(precision):
    cams, mets, gps, prims = _batch(precision)
    dt = _dtype(precision)
    direct = _outs(cams, dt)
    native.blacklight_launch_count(reset=True)
    assert native.blacklight_trace_batch(cams, mets, gps, prims, [FREQ] * 4, direct) == 0
    # camera frames, the prediction (block list, descriptors, initial states, centre-ray
    # geodesics, sort), then the wave: geodesics, the transfer's ray order (key, scan, scatter;
    # the FP64 sample pass makes the keys) and the transfer, and the rays' initial states in
    # the fast form
    launches = {native.BL_PREC_FAST: 12, native.BL_PREC_MIXED: 11, native.BL_PREC_FP64: 12}[precision]
    assert native.blacklight_launch_count() == launches
    assert float(sum(o["stokes"][0].double().sum() for o in direct)) > 0.0
    morton = _outs(cams, dt)
    plan = native.Plan(cams, mets, gps, prims, [FREQ] * 4, morton, config={"ray_order": 0})
    assert plan.config()["ray_order"] == 0
    plan.run()
    assert plan.check() == 0
    _same(direct, morton)
    plan.close()
    # a plan takes the work-ordered queue by default for such a batch
    outs = _outs(cams, dt)
    plan = native.Plan(cams, mets, gps, prims, [FREQ] * 4, outs)
    assert plan.config()["ray_order"] == 2
    native.blacklight_launch_count(reset=True)
    plan.run()
    assert plan.check() == 0
    assert native.blacklight_launch_count() == launches
    _same(direct, outs)
    plan.close()


def test_work_ordered_trace_in_waves():
    precision = native.BL_PREC_FAST
    cams, mets, gps, prims = _batch(precision)
    ref = _outs(cams, torch.float32)
    assert native.blacklight_trace_batch(cams, mets, gps, prims, [FREQ] * 4, ref) == 0
    full = native.blacklight_workspace_size(cams, mets)
    ws = torch.empty(full // 5, dtype=torch.uint8, device=DEV)
    outs = _outs(cams, torch.float32)
    assert native.blacklight_trace_batch(cams, mets, gps, prims, [FREQ] * 4, outs,
                                         workspace=ws) == 0
    _same(ref, outs)


def test_geodesics_only_path_matches_traced_end_states():
    """blacklight_geodesics on one 256x256 image (work-ordered) against the end states of the
    same camera traced in a Morton-ordered plan."""
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.94, 60.0, n=256)
    met = S.Metric(**{**met.__dict__, "precision": native.BL_PREC_FP64})
    geo = images.alloc_outputs(cam.n, torch.float64, device=DEV, end_state=True)
    assert native.blacklight_geodesics(cam, met, geo) == 0
    outs = _outs([cam], torch.float64, end_state=True)
    plan = native.Plan([cam], [met], [gp], [torch.from_numpy(prim).to(DEV)], [FREQ], outs,
                       config={"ray_order": 0})
    plan.run()
    assert plan.check() == 0
    _same([geo], outs, keys=("status", "steps", "end_state"))
    plan.close()


def test_work_order_needs_an_eligible_batch():
    # the same four images on plane-layout grids: Morton by default, order 2 refused
    cams, mets, gps, prims = _batch(native.BL_PREC_FAST, cells=False)
    outs = _outs(cams, torch.float32)
    plan = native.Plan(cams, mets, gps, prims, [FREQ] * 4, outs)
    assert plan.config()["ray_order"] == 0
    plan.close()
    with pytest.raises(native.BlacklightError):
        native.Plan(cams, mets, gps, prims, [FREQ] * 4, outs, config={"ray_order": 2})
    native.blacklight_launch_count(reset=True)
    assert native.blacklight_trace_batch(cams, mets, gps, prims, [FREQ] * 4, outs) == 0
    # camera frames, initial states, geodesics, transfer: no reordering at all
    assert native.blacklight_launch_count() == 4
    # three small images (fewer than 65536 rays): Morton by default, order 2 refused
    cams, mets, gps, prims = [], [], [], []
    for spin, inc in ((0.9, 17.0), (0.5, 60.0), (0.0, 90.0)):
        cam, met, gp, prim = S.workload_inputs("torus64_cam32", spin, inc, n=32)
        cams.append(cam)
        mets.append(S.Metric(**{**met.__dict__, "precision": native.BL_PREC_FAST}))
        gps.append(gp)
        prims.append(torch.from_numpy(prim).to(DEV))
    plan = native.Plan(cams, mets, gps, prims, [FREQ] * 3, _outs(cams, torch.float32))
    assert plan.config()["ray_order"] == 0
    plan.close()
    with pytest.raises(native.BlacklightError):
        native.Plan(cams, mets, gps, prims, [FREQ] * 3, _outs(cams, torch.float32),
                    config={"ray_order": 2})
