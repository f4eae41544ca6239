"""The positional split of the x-sorted rounds (Sec. 3, Sec. 4.4), checked in exact arithmetic on the CPU.

The sorted form keeps a segment's points in the chain's x order and splits the
segment at its farthest point C by position: a point before C is tested only
against h -> C, a point after C only against C -> e.  This model of the rounds
(rational arithmetic, no floating-point filter, no CUDA) checks on many small
sets -- with many equal x values, duplicates and points on the bounding box --
and under random orders of equal-x points that, in every round of both initial
splits:
  * the positional rule keeps exactly the points the two-test rule keeps
    (strictly right of h -> C, else strictly right of C -> e), each in the same
    child;
  * the children are contiguous runs before and after C;
and that the final heads are the monotone-chain oracle's hull with the
generation-synchronous oracle's live counts.  It pins the claim the CUDA kernels
rely on, independently of them.
"""
import numpy as np
import pytest

import oracle
import pins
from exact import dist_sign, orient


def _extremes(pts):
    n = len(pts)
    a = b = bot = top = 0
    for k in range(1, n):
        x, y = float(pts[k][0]), float(pts[k][1])
        if (x, y, k) < (float(pts[a][0]), float(pts[a][1]), a):
            a = k
        if (x, y, -k) > (float(pts[b][0]), float(pts[b][1]), -b):
            b = k
        if (y, x, k) < (float(pts[bot][1]), float(pts[bot][0]), bot):
            bot = k
        if (y, x, -k) > (float(pts[top][1]), float(pts[top][0]), -top):
            top = k
    return a, b, bot, top


def _same(pts, i, j):
    return float(pts[i][0]) == float(pts[j][0]) and float(pts[i][1]) == float(pts[j][1])


def _farther(pts, h, e, p, q):
    """p farther from chord h -> e than q: distance, then lexicographically smaller (x, y), then index."""
    s = dist_sign(pts[h], pts[e], pts[p], pts[q])
    if s:
        return s > 0
    if not _same(pts, p, q):
        return (float(pts[p][0]), float(pts[p][1])) < (float(pts[q][0]), float(pts[q][1]))
    return p < q


def sorted_rounds(pts, mode, rng):
    """Model of the x-sorted form; returns (hull indices, live counts per generation)."""
    n = len(pts)
    if n == 0:
        return [], []
    a, b, bot, top = _extremes(pts)
    if _same(pts, a, b):
        return [a], []
    poly = [a]
    if mode == "quad" and not _same(pts, bot, a) and not _same(pts, bot, b):
        poly.append(bot)
    ib = len(poly)
    poly.append(b)
    if mode == "quad" and not _same(pts, top, a) and not _same(pts, top, b):
        poly.append(top)
    K = len(poly)
    chains = ([], [])
    for j, v in enumerate(poly):
        chains[0 if j < ib else 1].append((v, True))
    live0 = 0
    for i in range(n):
        if i in poly:
            continue
        for j in range(K):
            if orient(pts[poly[j]], pts[poly[(j + 1) % K]], pts[i]) < 0:
                chains[0 if j < ib else 1].append((i, False))
                live0 += 1
                break
    # x order per chain (ascending, then descending), equal x in a random order
    order = []
    for c, sign in ((0, 1.0), (1, -1.0)):
        items = chains[c]
        perm = rng.permutation(len(items))
        items = [items[k] for k in perm]
        items.sort(key=lambda t: sign * float(pts[t[0]][0]))  # stable: ties keep the random order
        order += items
    assert order[0] == (a, True)
    live = [live0]
    while live[-1] > 0:
        heads = [k for k, t in enumerate(order) if t[1]]
        bounds = heads + [len(order)]
        new = []
        kept_points = 0
        for s, hpos in enumerate(heads):
            epos = bounds[s + 1]
            h = order[hpos][0]
            e = order[epos][0] if epos < len(order) else a
            run = [t[0] for t in order[hpos + 1:epos]]
            new.append(order[hpos])
            if not run:
                continue
            # every point of the run lies strictly right of its chord
            assert all(orient(pts[h], pts[e], pts[p]) < 0 for p in run)
            c = run[0]
            for p in run[1:]:
                if _farther(pts, h, e, p, c):
                    c = p
            cpos = run.index(c)
            left = [p for p in run[:cpos] if orient(pts[h], pts[c], pts[p]) < 0]
            right = [p for p in run[cpos + 1:] if orient(pts[c], pts[e], pts[p]) < 0]
            # the two-test rule over the whole run, with the child it assigns
            want_left = [p for p in run if p != c and orient(pts[h], pts[c], pts[p]) < 0]
            want_right = [p for p in run if p != c and orient(pts[h], pts[c], pts[p]) >= 0
                          and orient(pts[c], pts[e], pts[p]) < 0]
            assert left == want_left and right == want_right
            new += [(p, False) for p in left] + [(c, True)] + [(p, False) for p in right]
            kept_points += len(left) + len(right)
        order = new
        live.append(kept_points)
    return [t[0] for t in order], live


def _cases():
    rng = np.random.default_rng(21)
    cases = list(pins.small_random_sets(seed=23, count=60))
    for _ in range(30):  # coarse grids: many equal x, duplicates, points on the box
        k = int(rng.integers(2, 8))
        cases.append(rng.integers(0, k, size=(int(rng.integers(3, 120)), 2)).astype(np.float32))
    for _ in range(10):  # points on a circle with repeats, and a few inside
        t = rng.random(int(rng.integers(5, 80))) * 2 * np.pi
        c = np.stack([np.cos(t), np.sin(t)], 1).astype(np.float32)
        cases.append(np.concatenate([c, c[: len(c) // 3], (rng.random((7, 2)) - 0.5).astype(np.float32)]))
    cases.append(np.array([[0, 0], [0, 1], [0, 2], [1, 0], [1, 2], [2, 0], [2, 1], [2, 2], [1, 1]], np.float32))
    cases.append(np.array([[0.0, 0.0], [-0.0, 1.0], [0.0, -0.0], [-0.0, 2.0], [1.0, 1.0]], np.float32))
    return cases


@pytest.mark.parametrize("mode", ["quad", "chord"])
def test_positional_split_equals_two_test_rule(mode):
    rng = np.random.default_rng(7 if mode == "quad" else 8)
    for p in _cases():
        for _ in range(2):  # two random orders of equal-x points
            hull, live = sorted_rounds(p, mode, rng)
            assert hull == oracle.hull2d(p).tolist(), p.tolist()
            want_hull, want_live = oracle.quickhull(p, mode)
            assert hull == want_hull.tolist()
            assert live == want_live.tolist(), (p.tolist(), live, want_live.tolist())
