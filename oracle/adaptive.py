"""Oracle for adaptive ray tracing (Sec. 4, "Adaptive Ray Tracing") -- TEST INFRASTRUCTURE.

Plain Python on top of the oracle's tracer: a pixel of level L is a square of side w / (n 2^L)
sampled at its centre, which is exactly pixel (i, j) of an n 2^L camera, so each level traces
its blocks' pixels with that camera. Blocks are judged on their own pixels only.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import trace

ABS_GRAD, REL_GRAD, ABS_LAPL, REL_LAPL = 0, 1, 2, 3


def _diff1(line, crit):
    """First differences along a line of a block, one-sided at the ends."""
    B = line.size
    out = np.zeros(B)
    if B < 2:
        return out
    for w in range(B):
        if w == 0:
            lo, hi, central = 0, 1, False
        elif w == B - 1:
            lo, hi, central = B - 2, B - 1, False
        else:
            lo, hi, central = w - 1, w + 1, True
        if crit == ABS_GRAD:
            out[w] = 0.5 * (line[hi] - line[lo]) if central else line[hi] - line[lo]
        else:
            if central:
                den = line[lo] + 2.0 * line[w] + line[hi]
            else:
                den = line[lo] + line[hi]
            with np.errstate(divide="ignore", invalid="ignore"):
                out[w] = 2.0 * (line[hi] - line[lo]) / den
    return out


def _diff2(line, crit):
    """Second differences along a line, the stencil shifted inward at the ends."""
    B = line.size
    out = np.zeros(B)
    if B < 3:
        return out
    for w in range(B):
        c = min(max(w, 1), B - 2)
        lap = line[c - 1] - 2.0 * line[c] + line[c + 1]
        if crit == ABS_LAPL:
            out[w] = lap
        else:
            with np.errstate(divide="ignore", invalid="ignore"):
                out[w] = 4.0 * lap / (line[c - 1] + 2.0 * line[c] + line[c + 1])
    return out


def criterion_values(I, crit):
    """Criterion per pixel of a block I[v][u] (v = row j, u = column i)."""
    I = np.asarray(I, dtype=np.float64)
    B = I.shape[0]
    if crit in (ABS_GRAD, REL_GRAD):
        di = np.array([_diff1(I[v, :], crit) for v in range(B)])          # along i
        dj = np.array([_diff1(I[:, u], crit) for u in range(B)]).T        # along j
        return np.sqrt(di * di + dj * dj)
    di = np.array([_diff2(I[v, :], crit) for v in range(B)])
    dj = np.array([_diff2(I[:, u], crit) for u in range(B)]).T
    return np.abs(di + dj)


def _counted_values(I, crit, min_intensity):
    vals = criterion_values(I, crit)
    vals = np.where(np.asarray(I) >= min_intensity, vals, np.nan)   # faint pixels never count
    return vals


def refines(I, crit, threshold, min_count, min_intensity=0.0):
    vals = _counted_values(I, crit, min_intensity)
    with np.errstate(invalid="ignore"):
        return int(np.sum(vals > threshold)) >= min_count


def decision_margin(I, crit, threshold, min_count, min_intensity=0.0):
    """Relative distance of the deciding value (the min_count-th largest criterion value)
    from the threshold: how far the block is from flipping its refinement decision."""
    vals = np.sort(np.nan_to_num(_counted_values(I, crit, min_intensity), nan=-np.inf).ravel())[::-1]
    v = vals[min_count - 1]
    if not np.isfinite(v):
        return np.inf
    return abs(v - threshold) / abs(threshold)


def trace_adaptive(cam, met, gp, prim, freq, block, max_level, crit, threshold, min_count,
                   nthreads=0, margins=None, min_intensity=0.0):
    """Returns (composite [4][nf][nf], rays per level). If `margins` is a list, the decision
    margin of every judged block is appended to it."""
    n = cam.n
    nb = n // block
    blocks = [(bx, by) for by in range(nb) for bx in range(nb)]
    nf = n << max_level
    comp = np.zeros((4, nf, nf))
    level_rays = []
    for L in range(max_level + 1):
        nL = n << L
        level_rays.append(len(blocks) * block * block)
        if not blocks:
            break
        camL = dataclasses.replace(cam, n=nL)
        pix = np.array([(by * block + v) * nL + (bx * block + u) for bx, by in blocks
                        for v in range(block) for u in range(block)], dtype=np.int32)
        st = trace(camL, met, gp, prim, freq, pix=pix, nthreads=nthreads)["stokes"]
        s = 1 << (max_level - L)
        for p, px in enumerate(pix):
            j, i = divmod(int(px), nL)
            comp[:, j * s:(j + 1) * s, i * s:(i + 1) * s] = st[p][:, None, None]
        if L == max_level:
            break
        nxt = []
        b2 = block * block
        for b, (bx, by) in enumerate(blocks):
            I = st[b * b2:(b + 1) * b2, 0].reshape(block, block)
            if margins is not None:
                margins.append(decision_margin(I, crit, threshold, min_count, min_intensity))
            if refines(I, crit, threshold, min_count, min_intensity):
                for dy in range(2):
                    for dx in range(2):
                        nxt.append((2 * bx + dx, 2 * by + dy))
        blocks = nxt
    while len(level_rays) < max_level + 1:
        level_rays.append(0)
    return comp, np.array(level_rays)
