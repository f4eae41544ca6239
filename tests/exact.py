"""Exact-rational helpers for the tests: brute-force hulls and invariant checks.

Everything here uses Python's ``fractions.Fraction`` (or int64 where the values
are provably exact), so it is independent of both the C oracle's fixed-point
arithmetic and the CUDA path's floating-point filters.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np


def orient(a, b, c) -> int:
    """Exact sign of (bx-ax)(cy-ay) - (by-ay)(cx-ax) for float coordinates."""
    ax, ay = Fr(float(a[0])), Fr(float(a[1]))
    bx, by = Fr(float(b[0])), Fr(float(b[1]))
    cx, cy = Fr(float(c[0])), Fr(float(c[1]))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def dist_sign(u, v, p, q) -> int:
    """Exact sign of dist(p) - dist(q), dist(x) = -orient(u, v, x) (distance right of u->v)."""
    ux, uy = Fr(float(u[0])), Fr(float(u[1]))
    vx, vy = Fr(float(v[0])), Fr(float(v[1]))

    def dist(x):
        xx, xy = Fr(float(x[0])), Fr(float(x[1]))
        return -((vx - ux) * (xy - uy) - (vy - uy) * (xx - ux))

    d = dist(p) - dist(q)
    return (d > 0) - (d < 0)


def representatives(points) -> list[tuple[tuple[Fr, Fr], int]]:
    """Distinct coordinates (compared by value, -0 == +0) with their lowest index."""
    reps: dict[tuple[Fr, Fr], int] = {}
    for i, (x, y) in enumerate(np.asarray(points, dtype=np.float32)):
        key = (Fr(float(x)), Fr(float(y)))
        if key not in reps:
            reps[key] = i
    return list(reps.items())


def brute_hull(points) -> list[int]:
    """O(n^3) definition of the hull: strictly convex vertices, CCW from the lex-min point.

    (p, q) is a hull edge iff every point r satisfies orient(p, q, r) > 0, or
    orient(p, q, r) == 0 and r lies on the closed segment [p, q].  Collinear
    boundary points therefore never start an edge, and every vertex is
    represented by the lowest index among points with its coordinates.
    """
    reps = representatives(points)
    if not reps:
        return []
    if len(reps) == 1:
        return [reps[0][1]]
    coords = [k for k, _ in reps]

    def o(a, b, c):
        d = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        return (d > 0) - (d < 0)

    def on_segment(p, q, r):
        return (min(p[0], q[0]) <= r[0] <= max(p[0], q[0])) and (min(p[1], q[1]) <= r[1] <= max(p[1], q[1]))

    succ = {}
    for p in coords:
        for q in coords:
            if p == q:
                continue
            ok = True
            for r in coords:
                s = o(p, q, r)
                if s < 0 or (s == 0 and not on_segment(p, q, r)):
                    ok = False
                    break
            if ok:
                assert p not in succ, "hull successor must be unique"
                succ[p] = q
    start = min(succ)  # lexicographic (x, y) minimum among vertices
    assert start == min(coords)
    idx = dict(reps)
    out = [idx[start]]
    cur = succ[start]
    while cur != start:
        out.append(idx[cur])
        cur = succ[cur]
        assert len(out) <= len(coords)
    return out


def _orient_many_filtered(u, v, pts: np.ndarray) -> np.ndarray:
    """Exact signs of orient(u, v, p) for many p: float64 with a bound, rationals where unsure."""
    ux, uy, vx, vy = (np.float64(np.float32(t)) for t in (u[0], u[1], v[0], v[1]))
    px = pts[:, 0].astype(np.float64)
    py = pts[:, 1].astype(np.float64)
    # difference form in float64; each of the 7 roundings errs by at most 2^-53
    # relative, so 8 * 2^-53 * (|l| + |r|) bounds the error with margin
    l = (vx - ux) * (py - uy)
    r = (vy - uy) * (px - ux)
    s = l - r
    sign = np.sign(s).astype(np.int64)
    unsure = np.abs(s) <= (np.abs(l) + np.abs(r)) * 2.0 ** -50
    for k in np.nonzero(unsure)[0]:
        sign[k] = orient(u, v, pts[k])
    return sign


def check_hull_invariants(points, hull) -> None:
    """Assert that ``hull`` (indices) is the exact hull of ``points`` under the output rules.

    Holds at any size: containment (no point strictly right of any edge), strict
    convexity, a single CCW winding, start at the lexicographic minimum, and
    lowest-index representatives of distinct coordinates.
    """
    pts = np.asarray(points, dtype=np.float32)
    hull = [int(i) for i in hull]
    n = pts.shape[0]
    if n == 0:
        assert hull == []
        return
    order = np.lexsort((np.arange(n), pts[:, 1].astype(np.float64), pts[:, 0].astype(np.float64)))
    first = order[0]
    assert hull[0] == first, "hull must start at the lexicographically smallest point (lowest index)"
    # lowest-index representatives and distinct coordinates
    seen = set()
    for i in hull:
        key = (float(pts[i, 0]) + 0.0, float(pts[i, 1]) + 0.0)
        assert key not in seen, "duplicate vertex"
        seen.add(key)
        same = np.nonzero((pts[:, 0] == pts[i, 0]) & (pts[:, 1] == pts[i, 1]))[0]
        assert i == same.min(), "a vertex must be represented by its lowest index"
    h = len(hull)
    if h == 1:
        assert np.all((pts[:, 0] == pts[first, 0]) & (pts[:, 1] == pts[first, 1]))
        return
    if h == 2:
        a, b = pts[hull[0]], pts[hull[1]]
        sgn = _orient_many_filtered(a, b, pts)
        assert np.all(sgn == 0), "two-vertex hull requires all points collinear"
        # every point lies within the segment's bounding box
        lo = np.minimum(a, b)
        hi = np.maximum(a, b)
        assert np.all((pts >= lo) & (pts <= hi))
        return
    for k in range(h):
        u, v, w = pts[hull[k]], pts[hull[(k + 1) % h]], pts[hull[(k + 2) % h]]
        assert orient(u, v, w) > 0, "hull must be strictly convex and CCW"
    v0 = pts[hull[0]]
    for k in range(1, h - 1):
        assert orient(v0, pts[hull[k]], pts[hull[k + 1]]) > 0, "hull must wind once"
    for k in range(h):
        u, v = pts[hull[k]], pts[hull[(k + 1) % h]]
        sgn = _orient_many_filtered(u, v, pts)
        assert not np.any(sgn < 0), "a point lies strictly outside a hull edge"


def check_hull_int_grid(points, hull, scale: float) -> None:
    """Fast exact containment check when points * scale are integers below 2^30 (int64 arithmetic)."""
    p = np.round(np.asarray(points, dtype=np.float64) * scale).astype(np.int64)
    assert np.array_equal(p.astype(np.float64) / scale, np.asarray(points, dtype=np.float64))
    h = len(hull)
    for k in range(h):
        u = p[hull[k]]
        v = p[hull[(k + 1) % h]]
        o = (v[0] - u[0]) * (p[:, 1] - u[1]) - (v[1] - u[1]) * (p[:, 0] - u[0])
        assert not np.any(o < 0)
