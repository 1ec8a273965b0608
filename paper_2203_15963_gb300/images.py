"""Whole-image helpers over the C ABI: allocate torch outputs and call the binding."""
from __future__ import annotations

import torch

from . import native


def alloc_outputs(n: int, dtype=torch.float64, device="cuda", status=True, steps=True,
                  end_state=False, samples=False, aux=False):
    out = {"stokes": torch.empty((4, n, n), dtype=dtype, device=device)}
    if aux:
        out["aux"] = torch.empty((26, n, n), dtype=dtype, device=device)
    if samples:
        out["samples"] = torch.empty((n, n), dtype=torch.int32, device=device)
    if status:
        out["status"] = torch.empty((n, n), dtype=torch.int32, device=device)
    if steps:
        out["steps"] = torch.empty((n, n), dtype=torch.int32, device=device)
    if end_state:
        out["end_state"] = torch.empty((n, n, 8), dtype=torch.float64, device=device)
    return out


def trace_images(cams, mets, gps, prims, freqs, dtype=None, end_state=False, workspace=None,
                 flags=0, samples=False, outs=None, coef_mlp=None, aux=False):
    """Trace a batch of images in one launch pair; returns (rc, list of output dicts)."""
    if outs is None:
        outs = []
        for cam, met in zip(cams, mets):
            dt = dtype or (torch.float64 if met.precision == native.BL_PREC_FP64 else torch.float32)
            outs.append(alloc_outputs(cam.n, dt, end_state=end_state, samples=samples, aux=aux))
    rc = native.blacklight_trace_batch(cams, mets, gps, prims, freqs, outs, workspace=workspace,
                                       flags=flags, coef_mlp=coef_mlp)
    return rc, outs


def pack_grid(prim: torch.Tensor, gp):
    """The grid tensor `prim` (plane layout, on the device) repacked into the cell layout by
    the library; returns (cells tensor, grid parameters with layout = cells)."""
    import dataclasses
    n_snap = max(1, getattr(gp, "n_snapshots", 1))
    shape = (n_snap, gp.n_phi, gp.n_theta, gp.n_r, 8) if n_snap > 1 else \
        (gp.n_phi, gp.n_theta, gp.n_r, 8)
    cells = torch.empty(shape, dtype=torch.float32, device=prim.device)
    native.blacklight_grid_pack(prim, cells, gp)
    return cells, dataclasses.replace(gp, layout=native.BL_GRID_CELLS)
