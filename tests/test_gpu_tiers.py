"""Small-problem tiers at their limits, through the C ABI.

A set is built so that its four initial segments (the edges of the initial
quadrilateral A = (-1, 0), Bot = (0, -1), B = (1, 0), Top = (0, 1)) hold chosen
numbers of points: points on the unit circle strictly inside one quadrant lie
strictly right of that quadrant's edge only, and interior points are discarded
by the initial split.  With the 4096-point tile and cutover, segments of 1024
points (the largest finished in packs) and 1025 points (the smallest finished
alone) reach the block finisher, 4096 points (the cutover) too, and 4097 points
take a grid-wide round.  The hull and the per-generation live counts must equal
the oracle's.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _quadrant_set(counts, interior=3000, seed=0):
    rng = np.random.default_rng(seed)
    pts = [np.array([[-1.0, 0.0], [0.0, -1.0], [1.0, 0.0], [0.0, 1.0]], np.float32)]
    # quadrant of each edge: A->Bot (III), Bot->B (IV), B->Top (I), Top->A (II)
    for q, k in zip((2, 3, 0, 1), counts):
        t = q * np.pi / 2 + 0.01 + (np.pi / 2 - 0.02) * np.sort(rng.random(k))
        arc = np.stack([np.cos(t), np.sin(t)], 1).astype(np.float32)
        pts.append(arc)
    r = 0.5 * np.sqrt(rng.random(interior))
    a = 2 * np.pi * rng.random(interior)
    pts.append(np.stack([r * np.cos(a), r * np.sin(a)], 1).astype(np.float32))
    p = np.concatenate(pts)
    return p[rng.permutation(len(p))]


@pytest.mark.parametrize("counts", [(1024, 1025, 4096, 4097), (1, 1023, 1026, 5000), (17, 16, 1024, 1024)])
@pytest.mark.parametrize("mode", ["quad"])
def test_finisher_tier_limits(qh, counts, mode):
    import torch

    p = _quadrant_set(counts)
    want, live = oracle.quickhull(p, mode)
    assert np.array_equal(want, oracle.hull2d(p))
    plan = qh.Plan(len(p), 1)
    plan.set_tuning(4096)
    got = qh.hull2d(torch.from_numpy(p).cuda(), plan).cpu().numpy()
    st = plan.stats()
    assert st["device_status"] == 0
    assert np.array_equal(got, want)
    assert st["live"] == live.tolist()
    plan.close()
