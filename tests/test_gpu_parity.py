"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Index lists must match bit for bit: the hull is unique under the output rules,
so no tolerance applies.  Per-generation live counts must match the oracle's
generation-synchronous QuickHull exactly.
"""
import numpy as np
import pytest

import oracle
import pins
import synth
from exact import brute_hull, check_hull_invariants

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def plans(qh):
    ps = {}
    for mode in ("quad", "chord"):
        for prec in ("f32", "f64"):
            ps[(mode, prec)] = qh.Plan(2_000_000, 1, mode=qh.MODE_QUAD if mode == "quad" else qh.MODE_CHORD,
                                       prec=qh.PREC_F32 if prec == "f32" else qh.PREC_F64)
    yield ps
    for p in ps.values():
        p.close()


def _hull(qh, plan, pts):
    return qh.hull2d(_dev(pts), plan).cpu().numpy()


def test_device_predicates(qh):
    import torch
    from test_abi import _triples
    from exact import orient

    tri = _triples(seed=3)
    want = np.array([orient(t[0:2], t[2:4], t[4:6]) for t in tri])
    for prec in (0, 1):
        s, c = qh.check_orient_device(torch.from_numpy(tri).cuda(), prec)
        assert np.array_equal(s.cpu().numpy(), want)
        hs, hc = qh.check_orient_host(tri, prec)
        assert np.array_equal(c.cpu().numpy(), hc) or prec == 0  # host emulates directed rounding conservatively


def test_golden_and_small(qh, plans):
    cases = [pins.load_golden(p)[0] for p in pins.golden_cases()] + list(pins.small_random_sets(seed=9, count=120))
    for (mode, prec), plan in plans.items():
        for p in cases:
            want = brute_hull(p)
            got = _hull(qh, plan, p)
            assert got.tolist() == want, (mode, prec, p.tolist())


def test_empty_and_degenerate(qh, plans):
    plan = plans[("quad", "f32")]
    assert _hull(qh, plan, np.zeros((0, 2))).tolist() == []
    assert _hull(qh, plan, np.full((10, 2), 3.0)).tolist() == [0]
    big_same = np.full((300_000, 2), -1.5, dtype=np.float32)
    assert _hull(qh, plan, big_same).tolist() == [0]
    t = np.linspace(-1, 1, 100_001).astype(np.float32)
    line = np.stack([t, np.float32(0.5) * t], 1)
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(line))
    got = _hull(qh, plan, line[perm])
    assert got.tolist() == oracle.hull2d(line[perm]).tolist()
    assert len(got) == 2


def test_nonfinite_rejected(qh, plans):
    plan = plans[("quad", "f32")]
    for n in (50, 100_000):
        p = synth.disk(n)
        p[n // 3, 1] = np.nan
        with pytest.raises(qh.QhError) as e:
            _hull(qh, plan, p)
        assert e.value.status == 2
        p[n // 3, 1] = np.inf
        with pytest.raises(qh.QhError):
            _hull(qh, plan, p)


@pytest.mark.parametrize("name", ["square", "disk", "circle", "degenerate"])
@pytest.mark.parametrize("n", [4096, 4097, 6144, 10_001, 150_000])
def test_workloads_reduced(qh, plans, name, n):
    p = synth.make(name, n, seed=n)
    want = oracle.hull2d(p)
    for key, plan in plans.items():
        got = _hull(qh, plan, p)
        assert np.array_equal(got, want), (key, len(got), len(want))


@pytest.mark.parametrize("name", ["square", "disk", "circle", "degenerate"])
@pytest.mark.parametrize("mode", ["quad", "chord"])
def test_live_counts_match_oracle(qh, plans, name, mode):
    p = synth.make(name, 300_000, seed=2)
    plan = plans[(mode, "f32")]
    got = _hull(qh, plan, p)
    st = plan.stats()
    want_hull, want_live = oracle.quickhull(p, mode)
    assert np.array_equal(got, want_hull)
    assert st["device_status"] == 0
    assert st["generations"] == len(want_live)
    assert st["live"] == want_live.tolist()


def test_metamorphic_gpu(qh, plans):
    plan = plans[("quad", "f32")]
    p = synth.degenerate(400_000, grid=256)
    h = _hull(qh, plan, p)
    assert np.array_equal(_hull(qh, plan, p * np.float32(2.0 ** -20)), h)
    perm = np.random.default_rng(1).permutation(len(p))
    hp = _hull(qh, plan, p[perm])
    assert np.array_equal(p[perm][hp], p[h])


def test_batched_matches_per_set(qh):
    import torch

    p, off = synth.batched(300, seed=4, min_size=1, max_size=40_000)
    plan = qh.Plan(len(p), 300)
    out, counts = qh.hull2d_batched(_dev(p), torch.from_numpy(off).cuda(), plan)
    out = out.cpu().numpy()
    counts = counts.cpu().numpy()
    want_out, want_counts = oracle.hull2d_batched(p, off)
    assert np.array_equal(counts, want_counts)
    for s in range(len(counts)):
        a = int(off[s])
        assert np.array_equal(out[a:a + counts[s]], want_out[a:a + counts[s]]), s
    plan.close()


_FULL = {}


def _full(name, n=None):
    """A full-size workload and its oracle hull (the last one is kept for the next test)."""
    key = (name, n)
    if key not in _FULL:
        _FULL.clear()
        p = synth.make(name) if n is None else synth.make(name, n)
        _FULL[key] = (p, oracle.hull2d(p))
    return _FULL[key]


def test_config1_as_stated(qh):
    """Configuration 1 exactly: 100,000 points uniform in [0,1)^2 from seed 0, plain FP64 predicates
    (and the FP32 filtered form), bit-exact against the monotone-chain oracle."""
    p = synth.square()
    assert p.shape == (100_000, 2)
    want = oracle.hull2d(p)
    for prec in (qh.PREC_F64, qh.PREC_F32):
        for mode in (qh.MODE_QUAD, qh.MODE_CHORD):
            plan = qh.Plan(len(p), 1, mode=mode, prec=prec)
            assert np.array_equal(_hull(qh, plan, p), want), (mode, prec)
            assert plan.stats()["device_status"] == 0
            plan.close()


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["quad", "chord"])
@pytest.mark.parametrize("name", ["disk", "circle", "degenerate"])
def test_full_size(qh, name, mode):
    p, want = _full(name)
    plan = qh.Plan(len(p), 1, mode=qh.MODE_QUAD if mode == "quad" else qh.MODE_CHORD)
    got = _hull(qh, plan, p)
    assert np.array_equal(got, want), (len(got), len(want))
    plan.close()
    if mode == "quad":
        check_hull_invariants(p[:200_000], oracle.hull2d(p[:200_000]))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["disk", "circle", "degenerate"])
def test_full_size_plain_fp64(qh, name):
    """Configuration 2's plain-FP64 form (and the same form on configurations 3 and 4)."""
    p, want = _full(name)
    plan = qh.Plan(len(p), 1, prec=qh.PREC_F64)
    assert np.array_equal(_hull(qh, plan, p), want)
    plan.close()


@pytest.mark.slow
@pytest.mark.parametrize("n", [2_000_000, 20_000_000])
def test_square_sweep_sizes(qh, n):
    """The unit-square size sweep (Table 2 shapes) at 2M and 20M points, both initial splits."""
    p, want = _full("square", n)
    plan = qh.Plan(len(p), 1)
    for mode in (qh.MODE_QUAD, qh.MODE_CHORD):
        plan.set_flags(mode, qh.PREC_F32)
        assert np.array_equal(_hull(qh, plan, p), want), mode
    plan.close()


@pytest.mark.slow
def test_full_batched(qh):
    import torch

    p, off = synth.batched()
    plan = qh.Plan(len(p), len(off) - 1)
    out, counts = qh.hull2d_batched(_dev(p), torch.from_numpy(off).cuda(), plan)
    want_out, want_counts = oracle.hull2d_batched(p, off)
    assert np.array_equal(counts.cpu().numpy(), want_counts)
    out = out.cpu().numpy()
    for s in range(len(want_counts)):
        a = int(off[s])
        assert np.array_equal(out[a:a + want_counts[s]], want_out[a:a + want_counts[s]]), s
    plan.close()


def _lattice_polygon(radius: int) -> np.ndarray:
    """Vertices of a strictly convex lattice polygon (Jarnik's construction): the
    primitive integer vectors (a, b) with |a| + |b| <= radius, sorted by angle and
    summed.  Consecutive edges turn by a positive angle, so every vertex is a
    strict hull vertex; the coordinates stay integers below 2^24 (exact floats)."""
    import math

    vecs = [(a, b) for a in range(-radius, radius + 1) for b in range(-radius, radius + 1)
            if (a or b) and abs(a) + abs(b) <= radius and math.gcd(abs(a), abs(b)) == 1]
    vecs.sort(key=lambda v: math.atan2(v[1], v[0]))
    pts = np.cumsum(np.array(vecs, dtype=np.int64), axis=0)
    pts -= pts.min(axis=0)
    assert pts.max() < 1 << 24
    return pts.astype(np.float32)


def test_host_buffers(qh):
    """The host-buffer entry point: a small hull (count and indices read back
    together) and a hull of more vertices than that first read covers."""
    plan = qh.Plan(300_000, 1)
    rng = np.random.default_rng(5)
    small = rng.random((50_000, 2), dtype=np.float32)
    assert np.array_equal(qh.hull2d_host(small, plan), oracle.hull2d(small))
    ring = _lattice_polygon(260)                        # 82,400 strict vertices
    c = ring.mean(axis=0)
    inner = (c + (rng.random((100_000, 2)) - 0.5) * 1e5).astype(np.float32)  # well inside
    pts = np.concatenate([ring, inner])[rng.permutation(len(ring) + len(inner))]
    want = oracle.hull2d(pts)
    assert len(want) == len(ring) > 65536
    assert np.array_equal(qh.hull2d_host(pts, plan), want)
    plan.close()


def test_host_buffers_overlapped(qh):
    """The host-buffer entry point on sets of at least 11M points, where the copy of the
    second half overlaps the hull of the first, and the first half's vertices are hulled
    together with the second half: a disk of odd size, coordinate duplicates across the
    halves (the first half's indices must win), equal points, a circle, and a non-finite
    coordinate in the second half and in the first."""
    plan = qh.Plan(11_600_000, 1)
    disk = synth.disk(11_000_001, seed=12)
    assert np.array_equal(qh.hull2d_host(disk, plan), oracle.hull2d(disk))
    q = synth.disk(5_600_000, seed=13)
    twice = np.concatenate([q, q])
    got = qh.hull2d_host(twice, plan)
    assert np.array_equal(got, oracle.hull2d(twice)) and got.max() < len(q)
    same = np.full((11_100_000, 2), 0.75, dtype=np.float32)
    assert qh.hull2d_host(same, plan).tolist() == [0]
    ring = synth.circle(11_500_000, seed=14)
    assert np.array_equal(qh.hull2d_host(ring, plan), oracle.hull2d(ring))
    bad = synth.disk(11_500_000, seed=15)
    bad[11_000_000, 1] = np.nan
    with pytest.raises(qh.QhError) as e:
        qh.hull2d_host(bad, plan)
    assert e.value.status == 2
    bad[11_000_000, 1] = 0.0
    bad[10, 0] = np.inf
    with pytest.raises(qh.QhError) as e:
        qh.hull2d_host(bad, plan)
    assert e.value.status == 2
    small = synth.disk(100_000, seed=16)  # the direct path on the same plan afterwards
    assert np.array_equal(qh.hull2d_host(small, plan), oracle.hull2d(small))
    plan.close()


def test_batched_degenerate_sets(qh):
    """One batched call over sets of every kind the front end classifies: empty, a
    single point, equal points (small and tiled), a tiled collinear line, a circle,
    a strictly convex lattice polygon, and big sets next to tiny ones."""
    import torch

    rng = np.random.default_rng(11)
    t = np.linspace(-1, 1, 20_001).astype(np.float32)
    ring = _lattice_polygon(60)
    ang = rng.random(6000) * 2 * np.pi
    sets = [
        np.zeros((0, 2), np.float32),
        np.array([[0.25, -0.5]], np.float32),
        np.full((5, 2), 2.0, np.float32),
        np.full((10_000, 2), -1.5, np.float32),                                 # tiled, all equal
        np.stack([t, np.float32(0.5) * t], 1)[rng.permutation(len(t))],       # tiled, collinear
        np.zeros((0, 2), np.float32),
        np.stack([np.cos(ang), np.sin(ang)], 1).astype(np.float32),           # circle
        ring[rng.permutation(len(ring))],                                      # every point a vertex
        synth.disk(100_000, seed=3),
        np.array([[0, 0], [1, 0], [0, 1]], np.float32),
        rng.random((4097, 2), dtype=np.float32),
    ]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    p = np.concatenate(sets).astype(np.float32)
    plan = qh.Plan(len(p), len(sets))
    out, counts = qh.hull2d_batched(_dev(p), torch.from_numpy(off).cuda(), plan)
    out = out.cpu().numpy()
    counts = counts.cpu().numpy()
    want_out, want_counts = oracle.hull2d_batched(p, off)
    assert np.array_equal(counts, want_counts)
    assert want_counts[0] == 0 and want_counts[1] == 1 and want_counts[3] == 1 and want_counts[4] == 2
    assert want_counts[7] == len(ring)
    for s in range(len(sets)):
        a = int(off[s])
        assert np.array_equal(out[a:a + counts[s]], want_out[a:a + counts[s]]), s
    plan.close()
