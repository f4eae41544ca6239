"""Recursion depth and the device-side error paths, through the C ABI.

QuickHull's recursion depth is not bounded by a constant: on points in convex
position whose x-values spread over many orders of magnitude (synth.parabola)
every round splits a segment near the middle of its x-range and most points
stay in one child, so the grid-wide rounds run about 80 generations deep at one
million points.  The hull must still equal the oracle's, index for index, and
the per-generation live counts the generation-synchronous oracle's (Sec. 3-4.4).

The error paths are driven with the plan's debug limits, never with a faulting
input: a grid-barrier wait limited to one poll gives up (QH_ERR_TIMEOUT), and a
segment tree limited to a few nodes overflows (QH_ERR_CAPACITY).  Every wait of
the kernels is bounded, so both calls return; the same plan then computes the
exact hull again once the limits are reset.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

_CACHE = {}


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _parabola_oracle(n, mode):
    key = (n, mode)
    if key not in _CACHE:
        p = synth.parabola(n)
        _CACHE[key] = (p,) + oracle.quickhull(p, mode)
    return _CACHE[key]


@pytest.mark.parametrize("mode", ["quad", "chord"])
@pytest.mark.parametrize("block", [256, 128])
def test_deep_recursion_parabola(qh, mode, block):
    p, want, live = _parabola_oracle(1_000_000, mode)
    assert len(live) > 64  # deeper than any fixed level table of the earlier design
    assert np.array_equal(want, oracle.hull2d(p))
    plan = qh.Plan(len(p), 1, mode=qh.MODE_QUAD if mode == "quad" else qh.MODE_CHORD)
    plan.set_block(block)
    got = qh.hull2d(_dev(p), plan).cpu().numpy()
    st = plan.stats()
    assert st["device_status"] == 0
    assert np.array_equal(got, want), (len(got), len(want))
    assert st["generations"] == len(live)
    assert st["live"] == live.tolist()
    assert st["levels"] >= st["global_rounds"] + 1 > 64
    plan.close()


def test_deep_recursion_parabola_f64_and_batched(qh):
    """The same input in plain FP64, and as two sets of one batch next to a disk."""
    import torch

    p, want, _ = _parabola_oracle(1_000_000, "quad")
    plan = qh.Plan(len(p), 1, prec=qh.PREC_F64)
    assert np.array_equal(qh.hull2d(_dev(p), plan).cpu().numpy(), want)
    plan.close()
    q = synth.parabola(600_000, seed=3)
    d = synth.disk(300_000, seed=4)
    pts = np.concatenate([q, d, p]).astype(np.float32)
    off = np.array([0, len(q), len(q) + len(d), len(pts)], np.int64)
    plan = qh.Plan(len(pts), 3)
    out, counts = qh.hull2d_batched(_dev(pts), torch.from_numpy(off).cuda(), plan)
    out, counts = out.cpu().numpy(), counts.cpu().numpy()
    want_out, want_counts = oracle.hull2d_batched(pts, off)
    assert np.array_equal(counts, want_counts)
    for s in range(3):
        a = int(off[s])
        assert np.array_equal(out[a:a + counts[s]], want_out[a:a + counts[s]]), s
    plan.close()


@pytest.mark.slow
def test_deep_recursion_parabola_20m(qh):
    p = synth.parabola(20_000_000, seed=1)
    plan = qh.Plan(len(p), 1)
    got = qh.hull2d(_dev(p), plan).cpu().numpy()
    st = plan.stats()
    assert st["device_status"] == 0
    assert np.array_equal(got, oracle.hull2d(p))
    plan.close()


def test_grid_barrier_timeout_then_recovery(qh):
    p = synth.disk(1_000_000, seed=8)
    want = oracle.hull2d(p)
    d = _dev(p)
    plan = qh.Plan(len(p), 1)
    plan.set_debug(spin_limit=1)
    with pytest.raises(qh.QhError) as e:
        qh.hull2d(d, plan)
    assert e.value.status == 6  # QH_ERR_TIMEOUT, written to out_count as -6
    assert plan.stats()["device_status"] == 6
    plan.set_debug()
    assert np.array_equal(qh.hull2d(d, plan).cpu().numpy(), want)
    assert plan.stats()["device_status"] == 0
    plan.close()


def test_tree_capacity_error_then_recovery(qh):
    p, want, _ = _parabola_oracle(1_000_000, "quad")
    d = _dev(p)
    plan = qh.Plan(len(p), 1)
    plan.set_debug(max_tree_nodes=8)
    with pytest.raises(qh.QhError) as e:
        qh.hull2d(d, plan)
    assert e.value.status == 5  # QH_ERR_CAPACITY
    assert plan.stats()["device_status"] == 5
    plan.set_debug()
    assert np.array_equal(qh.hull2d(d, plan).cpu().numpy(), want)
    plan.close()
