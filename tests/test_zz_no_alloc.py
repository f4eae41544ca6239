"""The allocation-free entry point qh_hull2d_noalloc, through the C ABI.

It serves callers that must not allocate device memory at the moment they
need a hull: a real-time loop that cannot take cudaMalloc's implicit device
synchronisation, or a plug-in whose host application owns the device-memory
budget.  It takes its scratch from a fixed array in the library's device image
instead.  Its output must equal, index for index, both the plan-based entry
point's and the CPU oracle's (hulls are unique, so the tolerance is zero), on
consecutive calls that reuse the shared scratch, including the degenerate
cases (no points, one point, equal points, a non-finite coordinate) and an
input that recurses deeper than 64 generations.
This file is collected last, so a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.qh_hull2d_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call(fn, torch, p):
    """One call; returns the device count and the indices it reports."""
    t = torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).cuda().reshape(-1, 2)
    out = torch.full((max(len(p), 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    st = fn(t.data_ptr(), len(p), out.data_ptr(), cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    c = int(cnt.item())
    return c, (out[:c].cpu().numpy() if c > 0 else np.zeros(0, np.int32))


def test_noalloc_matches_plan_entry_point_and_oracle(qh):
    import torch

    fn = _noalloc(qh.load())
    cases = [synth.disk(200_000, seed=5), synth.degenerate(262_144, seed=6, grid=512),
             synth.circle(150_000, seed=7), synth.square(3000, seed=8), synth.parabola(262_144, seed=9),
             np.zeros((0, 2), np.float32), np.array([[0.5, -2.0]], np.float32),
             np.full((1000, 2), 3.25, np.float32)]
    plan = qh.Plan(262_144, 1)
    for p in cases + cases[:1]:  # consecutive calls, the last one repeating the first input
        want = oracle.hull2d(p)
        c, got = _call(fn, torch, p)
        assert c == len(want)
        assert np.array_equal(got, want)
        if len(p):
            assert np.array_equal(qh.hull2d(torch.from_numpy(p).cuda(), plan).cpu().numpy(), got)
    plan.close()


def test_noalloc_nonfinite_then_valid(qh):
    import torch

    fn = _noalloc(qh.load())
    p = synth.disk(50_000, seed=10)
    p[777, 0] = np.nan
    c, _ = _call(fn, torch, p)
    assert c == -2  # -QH_ERR_NONFINITE, written to out_count
    q = synth.disk(50_000, seed=11)
    c, got = _call(fn, torch, q)  # the next call on the same scratch is unaffected
    assert np.array_equal(got, oracle.hull2d(q))


def test_noalloc_rejects_oversize(qh):
    import torch

    fn = _noalloc(qh.load())
    t = torch.zeros((262_145, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros(262_145, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert fn(t.data_ptr(), 262_145, out.data_ptr(), cnt.data_ptr(),
              torch.cuda.current_stream().cuda_stream) == 5  # QH_ERR_CAPACITY
