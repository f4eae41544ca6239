"""Pins for the generation-synchronous QuickHull oracle (per-generation live counts).

The live count after each generation is the method's internal state (Sec. 4.4:
farthest point per segment, discard of the points inside triangle A-C-B).  It has
no closed form, so it is pinned by an independent pure-Python implementation with
exact rational arithmetic on small inputs, and by invariants at larger sizes.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import synth
from exact import brute_hull


def _py_quickhull(points, mode):
    """Pure-Python, exact-rational rounds: returns (hull, live counts)."""
    P = [(Fr(float(x)), Fr(float(y))) for x, y in np.asarray(points, dtype=np.float32)]
    n = len(P)

    def o(a, b, c):
        d = (P[b][0] - P[a][0]) * (P[c][1] - P[a][1]) - (P[b][1] - P[a][1]) * (P[c][0] - P[a][0])
        return (d > 0) - (d < 0)

    def dist(u, v, p):  # positive right of u->v
        return -((P[v][0] - P[u][0]) * (P[p][1] - P[u][1]) - (P[v][1] - P[u][1]) * (P[p][0] - P[u][0]))

    a = min(range(n), key=lambda i: (P[i][0], P[i][1], i))
    b = min(range(n), key=lambda i: (-P[i][0], -P[i][1], i))
    bot = min(range(n), key=lambda i: (P[i][1], P[i][0], i))
    top = min(range(n), key=lambda i: (-P[i][1], -P[i][0], i))
    if P[a] == P[b]:
        return [a], []
    poly = [a]
    if mode == "quad" and P[bot] not in (P[a], P[b]):
        poly.append(bot)
    poly.append(b)
    if mode == "quad" and P[top] not in (P[a], P[b]):
        poly.append(top)
    k = len(poly)
    segs = []
    for j in range(k):
        segs.append([poly[j], []])
    for i in range(n):
        for j in range(k):
            if o(poly[j], poly[(j + 1) % k], i) < 0:
                segs[j][1].append(i)
                break
    live = [sum(len(s[1]) for s in segs)]
    while any(s[1] for s in segs):
        new = []
        for j, (h, pts) in enumerate(segs):
            e = segs[(j + 1) % len(segs)][0]
            if not pts:
                new.append([h, []])
                continue
            c = min(pts, key=lambda p: (-dist(h, e, p), P[p][0], P[p][1], p))
            ac = [p for p in pts if o(h, c, p) < 0]
            cb = [p for p in pts if not o(h, c, p) < 0 and o(c, e, p) < 0]
            new += [[h, ac], [c, cb]]
        segs = new
        live.append(sum(len(s[1]) for s in segs))
    return [s[0] for s in segs], live


@pytest.mark.parametrize("mode", ["quad", "chord"])
def test_live_counts_match_pure_python(mode):
    rng = np.random.default_rng(11)
    for k in range(60):
        n = int(rng.integers(1, 60))
        if k % 3 == 0:
            p = rng.integers(0, 6, size=(n, 2)).astype(np.float32)
        elif k % 3 == 1:
            p = synth.disk(n, seed=k)
        else:
            p = synth.circle(n, seed=k, n_circle=n // 2)
        hull, live = oracle.quickhull(p, mode)
        want_hull, want_live = _py_quickhull(p, mode)
        assert hull.tolist() == want_hull
        assert live.tolist() == want_live
        assert hull.tolist() == brute_hull(p)


@pytest.mark.parametrize("name", ["square", "disk", "circle", "degenerate"])
def test_live_count_invariants(name):
    p = synth.make(name, 50000)
    for mode in ("quad", "chord"):
        hull, live = oracle.quickhull(p, mode)
        assert np.array_equal(hull, oracle.hull2d(p))
        assert live[-1] == 0 and live[0] <= len(p)
        # every generation removes at least the new vertex of each live segment
        assert np.all(np.diff(live) < 0)
    # the quadrilateral pre-step never keeps more points than the chord split
    _, lq = oracle.quickhull(p, "quad")
    _, lc = oracle.quickhull(p, "chord")
    assert lq[0] <= lc[0]
