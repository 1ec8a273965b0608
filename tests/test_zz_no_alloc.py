"""blacklight_trace_noalloc: the trace entry point for callers that cannot allocate device
memory (a fixed allocator budget, a foreign memory pool). It must give the same Stokes images
as blacklight_trace, call after call, while working only in its fixed in-library scratch.

This file is collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process."""
import ctypes
import math

import pytest
import torch

from paper_2203_15963_gb300 import images, native
from paper_2203_15963_gb300 import synth as S

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values (cuda.h): bytes of the pool in use now, and its high-water mark
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8


class _PoolWatch:
    """Device memory that cudaMalloc/cudaMallocAsync could take, read through the driver API:
    the device's free memory (any allocation lowers it) and the default memory pool's
    high-water mark (stream-ordered allocations raise it even when freed again)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _attr(self, a):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def snapshot(self):
        torch.cuda.synchronize()
        # reset the high-water mark to the current use (the driver accepts only 0, which sets it
        # to the current value)
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0
        return torch.cuda.mem_get_info()[0], self._attr(_USED_MEM_CURRENT)

    def check(self, snap):
        torch.cuda.synchronize()
        free0, used0 = snap
        assert self._attr(_USED_MEM_HIGH) == used0, "a stream-ordered allocation happened"
        assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed"


CASES = [
    # (camera, metric) pairs traced back to back; the second reuses the same scratch
    ("fp64_dp", native.BL_PREC_FP64,
     [dict(theta=17.0, n=32, integ=native.BL_INT_DP), dict(theta=60.0, n=24, integ=native.BL_INT_DP)]),
    ("mixed_dp", native.BL_PREC_MIXED,
     [dict(theta=17.0, n=32, integ=native.BL_INT_DP), dict(theta=60.0, n=24, integ=native.BL_INT_DP)]),
    # fixed-step RK2 at f_step = 0.02 from r = 1000 M: ~31 record chunks a ray in FP64, more than
    # one wave of 1024 rays holds in the array, so the rays run in several waves
    ("fp64_rk2", native.BL_PREC_FP64,
     [dict(theta=17.0, n=32, integ=native.BL_INT_RK2), dict(theta=60.0, n=32, integ=native.BL_INT_RK2)]),
]


@pytest.mark.parametrize("name,precision,calls", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_trace_on_consecutive_calls(name, precision, calls):
    native.build()
    native.load()
    gp = S.GridParams(n_r=64, n_theta=32, n_phi=32)
    prim = torch.from_numpy(S.make_torus(gp, 0.9, S.BASE_SEED)).cuda()
    dtype = torch.float64 if precision == native.BL_PREC_FP64 else torch.float32
    runs = []
    for c in calls:
        cam = S.Camera(theta=math.radians(c["theta"]), n=c["n"])
        met = S.Metric(spin=0.9, precision=precision, integrator=c["integ"], f_step=0.02)
        ref = images.alloc_outputs(cam.n, dtype)
        assert native.blacklight_trace(cam, met, gp, prim, 230e9, ref) == 0
        runs.append((cam, met, ref, images.alloc_outputs(cam.n, dtype)))
    # one call first: it loads the library's kernels on the device and looks up the array
    cam, met, _, got = runs[0]
    assert native.blacklight_trace_noalloc(cam, met, gp, prim, 230e9, got) == 0
    watch = _PoolWatch()
    snap = watch.snapshot()
    for cam, met, ref, got in runs:          # two calls in a row, no allocation around them
        got["stokes"].fill_(float("nan"))
        assert native.blacklight_trace_noalloc(cam, met, gp, prim, 230e9, got) == 0
    watch.check(snap)
    for cam, met, ref, got in runs:
        # the same kernels on the same rays: every ray is computed independently of the wave
        # it runs in, so the images are equal bit for bit
        assert torch.equal(got["status"], ref["status"])
        assert torch.equal(got["steps"], ref["steps"])
        assert torch.allclose(got["stokes"], ref["stokes"], rtol=0.0, atol=0.0, equal_nan=True)


def test_noalloc_rejects_cameras_beyond_its_scratch():
    native.load()
    gp = S.GridParams(n_r=8, n_theta=8, n_phi=8)
    prim = torch.zeros((8, 8, 8, 8), dtype=torch.float32, device="cuda")
    cam = S.Camera(n=33)
    out = images.alloc_outputs(33, torch.float32)
    with pytest.raises(native.BlacklightError) as ei:
        native.blacklight_trace_noalloc(cam, S.Metric(precision=1), gp, prim, 230e9, out)
    assert ei.value.code == -1 and "scratch" in str(ei.value)
