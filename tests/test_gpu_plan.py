"""Plans: a batched trace captured once in a CUDA graph and replayed. Replays, autotuned and
hand-set launch configurations all give the same per-ray results as blacklight_trace_batch
(each ray is computed independently of the launch shape and the ray order)."""
import numpy as np
import pytest
import torch

from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.build()
    native.load()
    assert torch.cuda.is_available()


def _batch(precision=native.BL_PREC_FAST):
    cams, mets, gps, prims = [], [], [], []
    for spin, inc, n in ((0.9, 17.0, 32), (0.5, 60.0, 48), (0.0, 90.0, 32)):
        cam, met, gp, prim = S.workload_inputs("torus64_cam32", spin, inc, n=n)
        cams.append(cam)
        mets.append(S.Metric(**{**met.__dict__, "precision": precision}))
        gps.append(gp)
        prims.append(torch.from_numpy(prim).to(DEV))
    return cams, mets, gps, prims


def _outs(cams, dtype=torch.float32):
    return [images.alloc_outputs(c.n, dtype, device=DEV, samples=True) for c in cams]


def _same(a, b):
    for x, y in zip(a, b):
        for k in ("stokes", "status", "steps", "samples"):
            assert torch.equal(x[k], y[k]), k


@pytest.mark.parametrize("precision", [native.BL_PREC_FAST, native.BL_PREC_FP64])
def test_plan_replay_equals_direct_batch(precision):
    cams, mets, gps, prims = _batch(precision)
    dt = torch.float64 if precision == native.BL_PREC_FP64 else torch.float32
    direct = _outs(cams, dt)
    rc = native.blacklight_trace_batch(cams, mets, gps, prims, [230e9] * 3, direct)
    assert rc == 0
    outs = _outs(cams, dt)
    plan = native.Plan(cams, mets, gps, prims, [230e9] * 3, outs)
    for _ in range(2):               # replays are repeatable
        for o in outs:
            o["stokes"].fill_(-1.0)
        native.blacklight_launch_count(reset=True)
        plan.run()
        assert plan.check() == 0
        # camera frames + one wave: geodesics and transfer, and the rays' initial states in the
        # fast form, or in the FP64 form the sample pass and the transport pass's order (key,
        # scan and scatter of a counting sort); these grids are in the plane layout, so the
        # fast form's transfer keeps the queue order
        assert native.blacklight_launch_count() == (7 if precision == native.BL_PREC_FP64 else 4)
        _same(outs, direct)
    plan.close()


def test_autotuned_and_row_major_plans_give_identical_results():
    cams, mets, gps, prims = _batch()
    ref = _outs(cams)
    native.blacklight_trace_batch(cams, mets, gps, prims, [230e9] * 3, ref)
    outs = _outs(cams)
    plan = native.Plan(cams, mets, gps, prims, [230e9] * 3, outs, autotune=True)
    cfg = plan.config()
    print("autotuned", cfg)
    assert cfg["ray_order"] in (0, 1) and cfg["geo_ctas_per_sm"] >= 1
    assert cfg["tr_ctas_per_sm"] >= 1 and cfg["run_ms"] > 0
    assert cfg["ilv_block"] == 0             # unequal images: no interleaving to tune
    plan.run()
    plan.check()
    _same(outs, ref)
    # a second autotuned plan of the same shape reuses the cached choice
    plan2 = native.Plan(cams, mets, gps, prims, [230e9] * 3, _outs(cams), autotune=True)
    assert plan2.config() == cfg
    outs3 = _outs(cams)
    plan3 = native.Plan(cams, mets, gps, prims, [230e9] * 3, outs3,
                        config={"ray_order": 1, "geo_ctas_per_sm": 1, "tr_ctas_per_sm": 2})
    c3 = plan3.config()
    assert c3["ray_order"] == 1 and c3["geo_ctas_per_sm"] == 1 and c3["tr_ctas_per_sm"] == 2
    plan3.run()
    plan3.check()
    _same(outs3, ref)
    for p in (plan, plan2, plan3):
        p.close()


def test_interleave_block_is_scheduling_only():
    """Equal images on cell-layout grids are queued interleaved in blocks of ilv_block rays of
    one image; every block size the autotuner may pick gives the same outputs bit for bit, and
    a batch that cannot interleave (unequal images) reports 0."""
    cams, mets, gps, prims = [], [], [], []
    for spin, inc in ((0.9, 17.0), (0.5, 60.0), (0.0, 90.0)):
        cam, met, gp, prim = S.workload_inputs("torus64_cam32", spin, inc, n=64)
        cells, gpc = images.pack_grid(torch.from_numpy(prim).to(DEV), gp)
        cams.append(cam)
        mets.append(S.Metric(**{**met.__dict__, "precision": native.BL_PREC_FAST}))
        gps.append(gpc)
        prims.append(cells)
    ref = _outs(cams)
    native.blacklight_trace_batch(cams, mets, gps, prims, [230e9] * 3, ref)
    for blk in (64, 256, 1024, 4096):
        outs = _outs(cams)
        plan = native.Plan(cams, mets, gps, prims, [230e9] * 3, outs, config={"ilv_block": blk})
        assert plan.config()["ilv_block"] == blk
        plan.run()
        assert plan.check() == 0
        _same(outs, ref)
        plan.close()
    # unequal images never interleave
    c2, m2, g2, p2 = _batch()
    plan = native.Plan(c2, m2, g2, p2, [230e9] * 3, _outs(c2), config={"ilv_block": 1024})
    assert plan.config()["ilv_block"] == 0
    plan.close()


def test_plan_sees_new_grid_contents_between_runs():
    cams, mets, gps, prims = _batch()
    outs = _outs(cams)
    plan = native.Plan(cams, mets, gps, prims, [230e9] * 3, outs)
    plan.run()
    plan.check()
    first = [o["stokes"].clone() for o in outs]
    for p in prims:
        p[0].mul_(2.0)                 # a new snapshot written in place: denser plasma
    plan.run()
    plan.check()
    ref = _outs(cams)
    native.blacklight_trace_batch(cams, mets, gps, prims, [230e9] * 3, ref)
    _same(outs, ref)
    assert not torch.equal(outs[0]["stokes"], first[0])
    plan.close()


def test_plan_rejects_bad_arguments():
    cams, mets, gps, prims = _batch()
    with pytest.raises(native.BlacklightError):
        native.Plan(cams, mets, gps, prims, [230e9] * 3, _outs(cams),
                    config={"ray_order": 7})
    bad = [S.Metric(**{**mets[0].__dict__, "tol_abs": 0.0})] + mets[1:]
    with pytest.raises(native.BlacklightError):
        native.Plan(cams, bad, gps, prims, [230e9] * 3, _outs(cams))
