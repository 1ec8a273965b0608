"""Cell-major grid layout (BL_GRID_CELLS): the pack kernel against a numpy transpose, and traces
from packed grids equal, bit for bit, the traces from the plane layout (the trilinear sums keep
their order) in every transfer variant; invalid layouts and pointers are rejected."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2203_15963_gb300 import coefmodel, images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.build()
    native.load()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("dims,n_snap", [((5, 3, 2), 1), ((64, 32, 32), 1), ((7, 4, 3), 3),
                                         ((1, 1, 1), 1), ((37, 5, 9), 2)])
def test_pack_matches_the_transpose(dims, n_snap):
    n_r, n_t, n_p = dims
    gp = S.GridParams(n_r=n_r, n_theta=n_t, n_phi=n_p, n_snapshots=n_snap)
    planes = np.random.default_rng(5).standard_normal((n_snap, 8, n_p, n_t, n_r)).astype(np.float32)
    src = torch.from_numpy(planes if n_snap > 1 else planes[0]).to(DEV)
    cells, gp2 = images.pack_grid(src, gp)
    torch.cuda.synchronize()
    want = np.moveaxis(planes, 1, -1)           # [s][phi][theta][r][8]
    assert np.array_equal(cells.cpu().numpy().reshape(want.shape), want)
    assert gp2.layout == native.BL_GRID_CELLS


def _trace_both(cam, met, gp, prim, flags=0, aux=False, coef_mlp=None):
    p = torch.from_numpy(np.ascontiguousarray(prim)).to(DEV)
    cells, gpc = images.pack_grid(p, gp)
    res = []
    for g, q in ((gp, p), (gpc, cells)):
        rc, outs = images.trace_images([cam], [met], [g], [q], [230e9], flags=flags, aux=aux,
                                       samples=True, coef_mlp=coef_mlp)
        torch.cuda.synchronize()
        assert rc == 0
        res.append(outs[0])
    return res


CASES = {
    "fp64": (native.BL_PREC_FP64, {}, 0, False),
    "mixed": (native.BL_PREC_MIXED, {}, 0, False),
    "fast": (native.BL_PREC_FAST, {}, 0, False),
    "fast_nearest": (native.BL_PREC_FAST, {"interp": 0}, 0, False),
    "fp64_nearest": (native.BL_PREC_FP64, {"interp": 0}, 0, False),
    "fast_unpolarized_aux": (native.BL_PREC_FAST, {}, native.BL_UNPOLARIZED, True),
    "fp64_aux": (native.BL_PREC_FP64, {}, 0, True),
}


@pytest.mark.parametrize("case", list(CASES))
def test_cell_layout_trace_equals_plane_layout(case):
    precision, gp_kw, flags, aux = CASES[case]
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 60.0)
    met = dataclasses.replace(met, precision=precision)
    gp = dataclasses.replace(gp, **gp_kw)
    a, b = _trace_both(cam, met, gp, prim, flags=flags, aux=aux)
    assert float(a["stokes"].abs().sum()) > 0.0
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("interp", [1, 0])
def test_cell_layout_slow_light_equals_plane_layout(interp):
    cam, met, gp, prim = S.workload_inputs("torus64_slow4_cam32", 0.9, 60.0)
    met = dataclasses.replace(met, precision=native.BL_PREC_FAST)
    gp = dataclasses.replace(gp, time_interp=interp)
    a, b = _trace_both(cam, met, gp, prim)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_cell_layout_with_learned_coefficients_equals_plane_layout():
    params, _ = coefmodel.train(seed=11, n=1 << 16, batch=4096, steps=200)
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 17.0)
    met = dataclasses.replace(met, precision=native.BL_PREC_FAST)
    a, b = _trace_both(cam, met, gp, prim, coef_mlp=params)
    assert torch.isfinite(a["stokes"]).all()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_cell_layout_in_a_plan():
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.5, 60.0)
    met = dataclasses.replace(met, precision=native.BL_PREC_FAST)
    p = torch.from_numpy(prim).to(DEV)
    cells, gpc = images.pack_grid(p, gp)
    ref = [images.alloc_outputs(cam.n, torch.float32, device=DEV)]
    native.blacklight_trace_batch([cam], [met], [gp], [p], [230e9], ref)
    outs = [images.alloc_outputs(cam.n, torch.float32, device=DEV)]
    plan = native.Plan([cam], [met], [gpc], [cells], [230e9], outs)
    plan.run()
    plan.check()
    assert torch.equal(outs[0]["stokes"], ref[0]["stokes"])
    plan.close()


def test_invalid_layouts_and_pointers_are_rejected():
    cam, met, gp, prim = S.workload_inputs("torus64_cam32", 0.9, 60.0)
    p = torch.from_numpy(prim).to(DEV)
    out = [images.alloc_outputs(cam.n, torch.float64, device=DEV)]
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_trace_batch([cam], [met], [dataclasses.replace(gp, layout=2)], [p],
                                      [230e9], out)
    assert ei.value.code == -1
    # cells must start on a 16-byte boundary
    big = torch.empty(p.numel() + 4, dtype=torch.float32, device=DEV)
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_trace_batch([cam], [met], [dataclasses.replace(gp, layout=1)],
                                      [big[1:]], [230e9], out)
    assert ei.value.code == -1
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_grid_pack(p, big[1:], gp)
    assert ei.value.code == -1
    # overlapping, host and zero-size arguments
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_grid_pack(big, big, gp)
    assert ei.value.code == -1
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_grid_pack(torch.from_numpy(prim), torch.empty_like(p), gp)
    assert ei.value.code == -1
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_grid_pack(p, torch.empty_like(p),
                                    dataclasses.replace(gp, n_r=0))
    assert ei.value.code == -1
