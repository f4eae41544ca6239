"""Parity of the x-sorted form of the rounds (qh_hull2d_sorted, Sec. 3 and Sec. 4.2-4.4) with the oracle.

The sorted form keeps every segment as a contiguous run of an x-sorted polygon
and splits it at its farthest point by position, with one orientation test per
point.  Its hull must equal the monotone-chain oracle's index for index, and its
per-generation live counts must equal the generation-synchronous oracle's in
both initial splits: the positional split keeps exactly the points the two-test
rule keeps, in the same children.
"""
import numpy as np
import pytest

import oracle
import pins
import synth
from exact import brute_hull

pytestmark = pytest.mark.gpu

FLAGS = [("quad", "f32"), ("quad", "f64"), ("chord", "f32"), ("chord", "f64")]


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def plans(qh):
    ps = {}
    for mode, prec in FLAGS:
        ps[(mode, prec)] = qh.Plan(1_100_000, 1, mode=qh.MODE_QUAD if mode == "quad" else qh.MODE_CHORD,
                                   prec=qh.PREC_F32 if prec == "f32" else qh.PREC_F64)
    yield ps
    for p in ps.values():
        p.close()


def _sorted(qh, plan, pts):
    return qh.hull2d_sorted(_dev(pts), plan).cpu().numpy()


def test_golden_and_small(qh, plans):
    cases = [pins.load_golden(p)[0] for p in pins.golden_cases()] + list(pins.small_random_sets(seed=19, count=120))
    for key, plan in plans.items():
        for p in cases:
            assert _sorted(qh, plan, p).tolist() == brute_hull(p), (key, p.tolist())


def test_empty_and_degenerate(qh, plans):
    for key, plan in plans.items():
        assert _sorted(qh, plan, np.zeros((0, 2))).tolist() == []
        assert _sorted(qh, plan, np.full((10, 2), 3.0)).tolist() == [0]
        assert _sorted(qh, plan, np.array([[1.0, 2.0], [1.0, 2.0], [-0.0, 0.0], [0.0, -0.0]])).tolist() == [2, 0]
        t = np.linspace(-1, 1, 100_001).astype(np.float32)
        line = np.stack([t, np.float32(0.5) * t], 1)[np.random.default_rng(0).permutation(len(t))]
        got = _sorted(qh, plan, line)
        assert got.tolist() == oracle.hull2d(line).tolist() and len(got) == 2, key
        vert = np.stack([np.zeros_like(t), t], 1)
        assert _sorted(qh, plan, vert).tolist() == oracle.hull2d(vert).tolist(), key


def test_nonfinite_rejected(qh, plans):
    plan = plans[("quad", "f32")]
    for n in (50, 100_000):
        p = synth.disk(n)
        p[n // 3, 0] = np.nan
        with pytest.raises(qh.QhError) as e:
            _sorted(qh, plan, p)
        assert e.value.status == 2
        p[n // 3, 0] = -np.inf
        with pytest.raises(qh.QhError):
            _sorted(qh, plan, p)
    # the plan still works afterwards
    p = synth.disk(1000)
    assert np.array_equal(_sorted(qh, plan, p), oracle.hull2d(p))


@pytest.mark.parametrize("name", ["square", "disk", "circle", "degenerate"])
@pytest.mark.parametrize("n", [4095, 4097, 10_001, 150_000])
def test_workloads_reduced(qh, plans, name, n):
    """Several tiles of the sort and of the rounds, with a ragged last tile."""
    p = synth.make(name, n, seed=n + 7)
    want = oracle.hull2d(p)
    for key, plan in plans.items():
        assert np.array_equal(_sorted(qh, plan, p), want), key
        assert np.array_equal(qh.hull2d(_dev(p), plan).cpu().numpy(), want), key


@pytest.mark.parametrize("name", ["square", "disk", "circle", "degenerate"])
@pytest.mark.parametrize("mode", ["quad", "chord"])
def test_live_counts_match_oracle(qh, plans, name, mode):
    p = synth.make(name, 300_000, seed=5)
    plan = plans[(mode, "f32")]
    got = _sorted(qh, plan, p)
    st = plan.stats()
    want_hull, want_live = oracle.quickhull(p, mode)
    assert np.array_equal(got, want_hull)
    assert st["device_status"] == 0
    assert st["generations"] == len(want_live)
    assert st["live"] == want_live.tolist()


def test_equal_x_and_duplicates(qh, plans):
    """Many points share each x (a coarse grid, with duplicates): the sort key is x
    alone, so equal-x points arrive in any order around every head."""
    rng = np.random.default_rng(3)
    g = rng.integers(0, 64, size=(200_000, 2)).astype(np.float32)
    g[:1000] = g[1000:2000]  # exact duplicates at other indices
    want = oracle.hull2d(g)
    for key, plan in plans.items():
        assert np.array_equal(_sorted(qh, plan, g), want), key
        assert plan.stats()["live"] == oracle.quickhull(g, key[0])[1].tolist(), key


def test_lattice_polygon(qh, plans):
    """82,400 strict vertices among 100,000 interior points."""
    from test_gpu_parity import _lattice_polygon

    rng = np.random.default_rng(5)
    ring = _lattice_polygon(260)
    c = ring.mean(axis=0)
    inner = (c + (rng.random((100_000, 2)) - 0.5) * 1e5).astype(np.float32)
    pts = np.concatenate([ring, inner])[rng.permutation(len(ring) + len(inner))]
    want = oracle.hull2d(pts)
    assert len(want) == len(ring)
    for key in (("quad", "f32"), ("chord", "f64")):
        assert np.array_equal(_sorted(qh, plans[key], pts), want), key


@pytest.mark.parametrize("mode", ["quad", "chord"])
def test_deep_recursion_parabola(qh, plans, mode):
    """About 80 generations at one million points (many batches of rounds)."""
    p = synth.parabola(1_000_000)
    want, live = oracle.quickhull(p, mode)
    assert len(live) > 64
    plan = plans[(mode, "f32")]
    got = _sorted(qh, plan, p)
    st = plan.stats()
    assert st["device_status"] == 0
    assert np.array_equal(got, want), (len(got), len(want))
    assert st["generations"] == len(live)
    assert st["live"] == live.tolist()


def test_same_as_plan_path_on_reuse(qh, plans):
    """The sorted form and the plan path alternate on one plan; every call is exact."""
    plan = plans[("quad", "f32")]
    for seed in range(3):
        p = synth.disk(500_000, seed=seed)
        want = oracle.hull2d(p)
        assert np.array_equal(_sorted(qh, plan, p), want)
        assert np.array_equal(qh.hull2d(_dev(p), plan).cpu().numpy(), want)
        assert np.array_equal(_sorted(qh, plan, p[: 1 + seed * 1000]), oracle.hull2d(p[: 1 + seed * 1000]))


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # the refused call leaves the capture empty
def test_errors(qh):
    """Argument errors return before any device work; a capturing stream is refused (the host reads the
    end flag between batches of rounds); the plan works normally afterwards."""
    import ctypes

    import torch

    lib = qh.load()
    plan = qh.Plan(1000, 1)
    p = synth.disk(2000, seed=3)
    with pytest.raises(qh.QhError) as e:
        _sorted(qh, plan, p)
    assert e.value.status == 5  # QH_ERR_CAPACITY: more points than the plan holds
    t = _dev(p[:1000])
    out = torch.empty(1000, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.qh_hull2d_sorted(plan.handle, t.data_ptr() + 4, 999, out.data_ptr(), cnt.data_ptr(), s) == 1
    assert lib.qh_hull2d_sorted(plan.handle, t.data_ptr(), -1, out.data_ptr(), cnt.data_ptr(), s) == 1
    assert lib.qh_hull2d_sorted(plan.handle, t.data_ptr(), 10, out.data_ptr(), None, s) == 1
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    status = []
    with torch.cuda.graph(graph, stream=stream):
        status.append(lib.qh_hull2d_sorted(plan.handle, t.data_ptr(), 1000, out.data_ptr(), cnt.data_ptr(),
                                           stream.cuda_stream))
    assert status == [8]  # QH_ERR_UNSUPPORTED while capturing
    assert np.array_equal(_sorted(qh, plan, p[:1000]), oracle.hull2d(p[:1000]))
    plan.close()


@pytest.mark.slow
@pytest.mark.parametrize("name", ["disk", "circle"])
def test_full_size(qh, name):
    p = synth.make(name)
    want = oracle.hull2d(p)
    plan = qh.Plan(len(p), 1)
    for mode in (qh.MODE_QUAD, qh.MODE_CHORD):
        plan.set_flags(mode, qh.PREC_F32)
        assert np.array_equal(_sorted(qh, plan, p), want), mode
    plan.close()
