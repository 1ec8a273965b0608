"""The benchmark step in the launch configuration the benchmark times: nine 256x256 images
(spins 0, 0.5, 0.94 x inclinations 17, 60, 90 deg) on the 256x128x128 torus, grids packed into
the cell layout, one batched call -- so the work-ordered queue, the transfer orders and starts
and (FP64) the compacted sample pass all run -- checked against the oracle on seeded pixels of
every image. Bounds as for the single-image full-size test: FP64 1e-7 relative L2 per Stokes
parameter, the FP32-transfer forms 1e-3; statuses equal; flux within 1e-4."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu
DEV = "cuda"
FREQ = 230e9
SPINS = (0.0, 0.5, 0.94)
INCS = (17.0, 60.0, 90.0)
PIX_PER_IMAGE = 384


@pytest.fixture(scope="module")
def batch():
    native.build()
    native.load()
    O.build()
    cams, mets, host, dev = [], [], [], []
    rng = np.random.default_rng(2024)
    for spin in SPINS:
        cells = None
        for inc in INCS:
            cam, met, gp, prim = S.workload_inputs("torus256_cam256", spin, inc)
            if cells is None:
                cells = images.pack_grid(torch.from_numpy(prim).to(DEV), gp)
            pix = np.sort(rng.choice(cam.n * cam.n, PIX_PER_IMAGE, replace=False)).astype(np.int32)
            cams.append(cam)
            mets.append(met)
            host.append((gp, prim, pix))
            dev.append(cells)
    oracle = [O.trace(c, m, gp, prim, FREQ, pix=pix) for c, m, (gp, prim, pix) in
              zip(cams, mets, host)]
    return cams, mets, host, dev, oracle


def _rel_l2(got, want):
    nI = np.linalg.norm(want[:, 0])
    return [float(np.linalg.norm(got[:, s] - want[:, s]) / nI) for s in range(4)]


@pytest.mark.parametrize("precision", [native.BL_PREC_FP64, native.BL_PREC_MIXED,
                                       native.BL_PREC_FAST])
def test_benchmark_batch_against_oracle(batch, precision):
    cams, mets, host, dev, oracle = batch
    mets = [S.Metric(**{**m.__dict__, "precision": precision}) for m in mets]
    dt = torch.float64 if precision == native.BL_PREC_FP64 else torch.float32
    outs = [images.alloc_outputs(c.n, dt, device=DEV) for c in cams]
    rc = native.blacklight_trace_batch(cams, mets, [d[1] for d in dev], [d[0] for d in dev],
                                       [FREQ] * len(cams), outs)
    torch.cuda.synchronize()
    assert rc == 0
    bound = 1e-7 if precision == native.BL_PREC_FP64 else 1e-3
    for q, ((gp, prim, pix), ora) in enumerate(zip(host, oracle)):
        st = outs[q]["stokes"].double().cpu().numpy().reshape(4, -1).T[pix]
        err = _rel_l2(st, ora["stokes"])
        print("image", q, "precision", precision, "rel-L2", err)
        assert max(err) <= bound, (q, err)
        assert abs(np.sum(st[:, 0]) / np.sum(ora["stokes"][:, 0]) - 1) <= 1e-4
        status = outs[q]["status"].cpu().numpy().reshape(-1)[pix]
        assert np.array_equal(status, ora["status"])
