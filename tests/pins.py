"""Pin checks for the CPU oracle, shared by the pin tests and the planted-mistake tests.

Each check raises AssertionError on a mismatch.  They compare the oracle with
things other than itself: exact rational arithmetic (``fractions.Fraction``), an
O(n^3) brute-force hull, hand-derived fixtures (``tests/golden``), closed forms,
invariants and metamorphic relations.
"""
from __future__ import annotations

import glob
import os

import numpy as np

import oracle
from exact import brute_hull, check_hull_invariants, dist_sign, orient

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(path):
    pts, hull = [], None
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "p":
                pts.append((float(tok[1]), float(tok[2])))
            elif tok[0] == "hull":
                hull = [int(t) for t in tok[1:]]
    return np.array(pts, dtype=np.float32).reshape(-1, 2), hull


def golden_cases():
    return sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


def adversarial_triples(rng, count=400):
    """Near-collinear and wide-dynamic-range triples, plus exact collinear ones."""
    out = [
        # exactly collinear, but naive double summation of the six products is wrong
        ((1.0, 2.0 ** -10), (1.0, 5.0), (1.0, 2.0 ** 60)),
        ((0.0, 0.0), (2.0, 2.0), (1.0, 1.0 + 2.0 ** -23)),
        ((0.0, 0.0), (2.0, 2.0), (1.0, 1.0)),
        ((0.0, 0.0), (-0.0, 1.0), (0.0, 2.0)),
        ((2.0 ** -149, 0.0), (0.0, 2.0 ** -149), (2.0 ** -148, -(2.0 ** -149))),
        ((1e30, 1e30), (-1e30, -1e30), (3e29, 3e29)),
        ((3.0e38, 1.0), (-3.0e38, -1.0), (0.0, 0.0)),
    ]
    for _ in range(count):
        s = np.float32(2.0 ** int(rng.integers(-30, 40)))
        a = (rng.random(2) * s).astype(np.float32)
        d = ((rng.random(2) - 0.5) * s).astype(np.float32)
        t = np.float32(rng.random() * 3 - 1)
        b = (a + d).astype(np.float32)
        c = (a + d * t).astype(np.float32)
        k = int(rng.integers(-2, 3))
        c = np.array([c[0], np.nextafter(c[1], np.float32(np.inf if k > 0 else -np.inf)) if k else c[1]],
                     dtype=np.float32)
        out.append((tuple(a.tolist()), tuple(b.tolist()), tuple(c.tolist())))
    return out


def check_orient(mutation=0, seed=0):
    rng = np.random.default_rng(seed)
    for a, b, c in adversarial_triples(rng):
        want = orient(a, b, c)
        got = oracle.orient_sign(a, b, c, mutation=mutation)
        assert got == want, (a, b, c, got, want)
        assert oracle.orient_sign(a, b, c, always_exact=True, mutation=mutation) == want
    for _ in range(2000):
        p = rng.integers(-4, 5, size=(3, 2)).astype(np.float32) / np.float32(4)
        assert oracle.orient_sign(*p, mutation=mutation) == orient(*p)


def check_dist_cmp(mutation=0, seed=0):
    rng = np.random.default_rng(seed)
    for _ in range(1500):
        q = rng.integers(-6, 7, size=(4, 2)).astype(np.float32)
        assert oracle.dist_cmp(*q, mutation=mutation) == dist_sign(*q)
    for _ in range(500):
        s = np.float32(2.0 ** int(rng.integers(-20, 30)))
        q = (rng.random((4, 2)) * s).astype(np.float32)
        q[3] = q[2]
        q[3, 1] = np.nextafter(q[3, 1], np.float32(np.inf))
        assert oracle.dist_cmp(*q, mutation=mutation) == dist_sign(*q)


def check_golden(mutation=0):
    for path in golden_cases():
        pts, hull = load_golden(path)
        assert oracle.hull2d(pts, mutation=mutation).tolist() == hull, path
        assert brute_hull(pts) == hull, path
        for mode in ("quad", "chord"):
            got, _ = oracle.quickhull(pts, mode, mutation=mutation)
            assert got.tolist() == hull, (path, mode)


def small_random_sets(seed=0, count=300):
    rng = np.random.default_rng(seed)
    for k in range(count):
        n = int(rng.integers(1, 13))
        kind = k % 4
        if kind == 0:  # tiny integer grid: duplicates and collinear points
            p = rng.integers(0, 4, size=(n, 2)).astype(np.float32)
        elif kind == 1:  # random floats
            p = rng.random((n, 2), dtype=np.float32)
        elif kind == 2:  # near a line, +-1 ulp
            x = rng.random(n).astype(np.float32)
            y = (np.float32(0.3) * x).astype(np.float32)
            step = rng.integers(-1, 2, size=n)
            y = np.where(step > 0, np.nextafter(y, np.float32(2)), np.where(step < 0, np.nextafter(y, np.float32(-2)), y))
            p = np.stack([x, y.astype(np.float32)], axis=1)
        else:  # signed grid with -0 and duplicates
            p = (rng.integers(-2, 3, size=(n, 2)).astype(np.float32) * np.float32(0.5))
            p[rng.random(n) < 0.2] *= np.float32(-1)
        yield p.astype(np.float32)


def check_brute_random(mutation=0, seed=0):
    for p in small_random_sets(seed):
        want = brute_hull(p)
        assert oracle.hull2d(p, mutation=mutation).tolist() == want, p.tolist()
        for mode in ("quad", "chord"):
            got, _ = oracle.quickhull(p, mode, mutation=mutation)
            assert got.tolist() == want, (mode, p.tolist())


def check_grid_subsets(mutation=0):
    """Every subset of the 3x3 grid {0,1,2}^2 (with one duplicated point each)."""
    grid = [(x, y) for x in range(3) for y in range(3)]
    for mask in range(1, 1 << 9):
        sub = [grid[i] for i in range(9) if mask >> i & 1]
        sub = sub + sub[:1]  # duplicate of the first point, at the highest index
        p = np.array(sub[::-1], dtype=np.float32)  # reversed: the duplicate comes first
        want = brute_hull(p)
        assert oracle.hull2d(p, mutation=mutation).tolist() == want, sub
        got, _ = oracle.quickhull(p, "quad", mutation=mutation)
        assert got.tolist() == want, sub


def check_closed_forms(mutation=0):
    h = lambda p: oracle.hull2d(np.asarray(p, dtype=np.float32), mutation=mutation).tolist()
    assert h(np.zeros((0, 2))) == []
    assert h([[3, 3]] * 5) == [0]
    assert h([[1, 1], [0, 0], [1, 1], [0, 0]]) == [1, 0]
    # all collinear: the two endpoints, lex-min first
    t = np.linspace(-3, 5, 17).astype(np.float32)
    assert h(np.stack([t[::-1], np.float32(2) * t[::-1]], 1)) == [16, 0]
    # regular lattice octagon plus interior points, shuffled
    octagon = [(-1, -2), (1, -2), (2, -1), (2, 1), (1, 2), (-1, 2), (-2, 1), (-2, -1)]
    inner = [(0, 0), (1, 1), (-1, 0), (0, -2), (2, 0)]  # (0,-2) and (2,0) lie on edges
    pts = octagon + inner
    perm = np.random.default_rng(7).permutation(len(pts))
    p = np.array([pts[i] for i in perm], dtype=np.float32)
    pos = {tuple(map(int, p[i])): i for i in range(len(p))}
    start = octagon.index((-2, -1))
    want = [pos[octagon[(start + k) % 8]] for k in range(8)]
    assert h(p) == want


def check_invariants_medium(mutation=0, seed=0):
    import synth

    for name, n in (("square", 20000), ("disk", 20000), ("circle", 20000), ("degenerate", 20000)):
        p = synth.make(name, n, seed=seed)
        hull = oracle.hull2d(p, mutation=mutation)
        check_hull_invariants(p, hull)
        for mode in ("quad", "chord"):
            got, live = oracle.quickhull(p, mode, mutation=mutation)
            assert np.array_equal(got, hull), (name, mode)


def check_metamorphic(mutation=0, seed=0):
    import synth

    rng = np.random.default_rng(seed)
    p = synth.degenerate(5000, seed=seed, grid=64)
    hull = oracle.hull2d(p, mutation=mutation)
    # scaling by a power of two is exact: same indices
    for k in (-7, 5):
        assert np.array_equal(oracle.hull2d(p * np.float32(2.0 ** k), mutation=mutation), hull)
    # a permutation maps vertices to the same coordinates (representatives may change)
    perm = rng.permutation(p.shape[0])
    hp = oracle.hull2d(p[perm], mutation=mutation)
    assert np.array_equal(p[perm][hp], p[hull])
    # mirroring x -> -x reverses the cyclic order
    q = p.copy()
    q[:, 0] = -q[:, 0]
    hm = oracle.hull2d(q, mutation=mutation)
    ring = list(hull[::-1])
    start = ring.index(hm[0])
    assert list(hm) == ring[start:] + ring[:start]


def check_batched(mutation=0):
    import synth

    p, off = synth.batched(24, seed=3, min_size=1, max_size=3000)
    out, counts = oracle.hull2d_batched(p, off)
    for s in range(len(counts)):
        a, b = int(off[s]), int(off[s + 1])
        want = oracle.hull2d(p[a:b], mutation=mutation)
        assert counts[s] == len(want)
        assert np.array_equal(out[a:a + counts[s]], want)


ALL_CHECKS = [check_orient, check_dist_cmp, check_golden, check_brute_random, check_grid_subsets,
              check_closed_forms, check_invariants_medium, check_metamorphic]


def run_all(mutation):
    """Run every check against an oracle variant; return the names of the checks that failed."""
    failed = []
    for chk in ALL_CHECKS:
        try:
            chk(mutation=mutation)
        except (AssertionError, oracle.OracleError):
            failed.append(chk.__name__)
    return failed

