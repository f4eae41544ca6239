"""The allocation-free entry point qh_hull2d_noalloc, through the C ABI.

It serves callers that must not allocate device memory when they need a hull
(real-time loops, plug-ins whose host owns the device-memory budget); it takes
its scratch from a fixed array in the library's device image.  Its output must
equal the plan-based entry point's, index for index (hulls are unique, so the
tolerance is zero), on consecutive calls that reuse the shared scratch.
This file is collected last, so a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.qh_hull2d_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_matches_plan_entry_point(qh):
    import torch

    lib = qh.load()
    fn = _noalloc(lib)
    cases = [synth.disk(200_000, seed=5), synth.degenerate(262_144, seed=6, grid=512),
             synth.circle(150_000, seed=7), synth.square(3000, seed=8)]
    plan = qh.Plan(262_144, 1)
    stream = torch.cuda.current_stream().cuda_stream
    for p in cases + cases[:1]:  # consecutive calls, the last one repeating the first input
        t = torch.from_numpy(p).cuda()
        want = qh.hull2d(t, plan).cpu().numpy()
        out = torch.full((len(p),), -7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert fn(t.data_ptr(), len(p), out.data_ptr(), cnt.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        c = int(cnt.item())
        assert c == len(want)
        assert np.array_equal(out[:c].cpu().numpy(), want)
    plan.close()


def test_noalloc_rejects_oversize(qh):
    import torch

    fn = _noalloc(qh.load())
    t = torch.zeros((262_145, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros(262_145, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert fn(t.data_ptr(), 262_145, out.data_ptr(), cnt.data_ptr(),
              torch.cuda.current_stream().cuda_stream) == 5  # QH_ERR_CAPACITY
