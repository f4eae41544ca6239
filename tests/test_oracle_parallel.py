"""The all-core driver of the CPU baseline gives the single-thread oracle's hull.

It hulls contiguous chunks in threads and then the union of the chunk hulls; the
cases put hull vertices, duplicates of them (the lowest index must win) and
collinear boundary points in different chunks, and cover the paths that fall
back to one thread.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("name,n", [("disk", 300_000), ("circle", 200_000), ("degenerate", 400_000),
                                    ("square", 100_000), ("parabola", 200_000)])
@pytest.mark.parametrize("threads", [2, 3, 8])
def test_parallel_equals_single_thread(name, n, threads):
    p = synth.make(name, n)
    assert np.array_equal(oracle.hull2d_parallel(p, threads), oracle.hull2d(p))


def test_duplicated_vertices_across_chunks_keep_lowest_index():
    rng = np.random.default_rng(3)
    base = rng.random((50_000, 2), dtype=np.float32)
    p = np.concatenate([base, base[::-1], base])  # every point three times, in three different chunks
    got = oracle.hull2d_parallel(p, 6)
    assert np.array_equal(got, oracle.hull2d(p))
    assert got.max() < len(base)  # the first copy of every vertex


def test_collinear_boundary_across_chunks():
    x = np.arange(60_000, dtype=np.float32)
    p = np.concatenate([np.stack([x, np.zeros_like(x)], 1), np.stack([x, np.full_like(x, 7.0)], 1)])
    perm = np.random.default_rng(4).permutation(len(p))
    p = p[perm]
    got = oracle.hull2d_parallel(p, 5)
    assert np.array_equal(got, oracle.hull2d(p))
    assert len(got) == 4


def test_small_inputs_and_errors():
    for p in [np.zeros((0, 2), np.float32), np.array([[1.0, 2.0]], np.float32), synth.disk(5000, seed=2)]:
        assert np.array_equal(oracle.hull2d_parallel(p, 8), oracle.hull2d(p))
    p = synth.disk(200_000, seed=9)
    p[150_000, 1] = np.inf
    with pytest.raises(oracle.OracleError) as e:
        oracle.hull2d_parallel(p, 4)
    assert e.value.status == oracle.NONFINITE
