"""Seeded synthetic point sets for the 2D convex-hull workloads.

This module only draws random numbers; it holds none of the hull arithmetic.
Both the CUDA path and the CPU oracle are fed from here, so the two sides
always see byte-identical inputs.

Every generator uses NumPy's PCG64 seeded from ``SeedSequence([config_id, seed])``.
Uniform FP32 values come from ``rng.random(dtype=np.float32)`` (multiples of
2^-24); every other value is computed in float64 and rounded to float32 once.

Workloads (sizes are the defaults; every generator takes a smaller ``n`` for
tests):

1. ``square``  -- i.i.d. uniform in [0,1)^2, n = 100,000 (the shape of the
   first row of the paper's Table 2, unit-square point sets).
2. ``disk``    -- i.i.d. uniform in the unit disk (r = sqrt(U), angle = 2*pi*U),
   n = 20,000,000.
3. ``circle``  -- 1,000,000 points on the unit circle (angle uniform, coordinates
   rounded to FP32) plus 19,000,000 uniform in the disk of radius 0.999, shuffled.
4. ``degenerate`` -- 15,800,000 i.i.d. integer-grid points in {0..4095}^2 stored as
   FP32 (exact duplicates occur naturally, about a third of them) plus 200,000
   points on the line y = 0.1*x: x uniform FP32 in [-2048, 6144), y = fl32(0.1f*x)
   moved by -1, 0 or +1 ulp with equal probability; shuffled.
5. ``batched`` -- 4096 independent sets, size floor(64 * 4096^U) clamped to
   [64, 262144], each drawn uniform-square, uniform-disk or standard-Gaussian with
   equal probability; CSR int64 offsets.

Stress input (not one of the five workloads):

6. ``parabola`` -- points in convex position on y = x^2 with x = fl32(U^100):
   the x-values spread over dozens of binary orders of magnitude, so every
   QuickHull round splits a segment near the middle of its x-range and most of
   its points stay in one child; at 1,000,000 points the recursion runs about
   80 generations deep (a third of the points underflow to the origin).
"""
from __future__ import annotations

import numpy as np

CONFIG_IDS = {"square": 1, "disk": 2, "circle": 3, "degenerate": 4, "batched": 5, "parabola": 6}

FULL_SIZES = {
    "square": 100_000,
    "disk": 20_000_000,
    "circle": 20_000_000,
    "degenerate": 16_000_000,
    "batched": 4096,  # number of sets
    "parabola": 1_000_000,
}


def _rng(config_id: int, seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([config_id, seed])))


def _disk(rng: np.random.Generator, n: int, radius: float = 1.0) -> np.ndarray:
    r = radius * np.sqrt(rng.random(n))
    t = 2.0 * np.pi * rng.random(n)
    out = np.empty((n, 2), dtype=np.float32)
    out[:, 0] = r * np.cos(t)
    out[:, 1] = r * np.sin(t)
    return out


def square(n: int = FULL_SIZES["square"], seed: int = 0) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^2 as float32[n, 2]."""
    rng = _rng(CONFIG_IDS["square"], seed)
    return rng.random((n, 2), dtype=np.float32)


def disk(n: int = FULL_SIZES["disk"], seed: int = 0) -> np.ndarray:
    """n points i.i.d. uniform in the unit disk as float32[n, 2]."""
    return _disk(_rng(CONFIG_IDS["disk"], seed), n)


def circle(n: int = FULL_SIZES["circle"], seed: int = 0, n_circle: int | None = None) -> np.ndarray:
    """n points: n/20 on the unit circle, the rest uniform in the disk of radius 0.999."""
    rng = _rng(CONFIG_IDS["circle"], seed)
    if n_circle is None:
        n_circle = n // 20
    t = 2.0 * np.pi * rng.random(n_circle)
    ring = np.empty((n_circle, 2), dtype=np.float32)
    ring[:, 0] = np.cos(t)
    ring[:, 1] = np.sin(t)
    inner = _disk(rng, n - n_circle, radius=0.999)
    pts = np.concatenate([ring, inner])
    return pts[rng.permutation(n)]


def degenerate(n: int = FULL_SIZES["degenerate"], seed: int = 0, n_line: int | None = None,
               grid: int = 4096) -> np.ndarray:
    """Integer grid {0..grid-1}^2 with natural duplicates plus near-line points y = 0.1 x (+-1 ulp)."""
    rng = _rng(CONFIG_IDS["degenerate"], seed)
    if n_line is None:
        n_line = max(1, n // 80)
    n_grid = n - n_line
    g = rng.integers(0, grid, size=(n_grid, 2)).astype(np.float32)
    lo, hi = -0.5 * grid, 1.5 * grid
    x = (lo + (hi - lo) * rng.random(n_line)).astype(np.float32)
    y = (np.float32(0.1) * x).astype(np.float32)
    step = rng.integers(-1, 2, size=n_line)
    y = np.where(step > 0, np.nextafter(y, np.float32(np.inf)),
                 np.where(step < 0, np.nextafter(y, np.float32(-np.inf)), y)).astype(np.float32)
    line = np.stack([x, y], axis=1)
    pts = np.concatenate([g, line])
    return pts[rng.permutation(n)]


def batched(num_sets: int = FULL_SIZES["batched"], seed: int = 0, min_size: int = 64,
            max_size: int = 262144) -> tuple[np.ndarray, np.ndarray]:
    """CSR batch: (float32[N, 2] points, int64[num_sets + 1] offsets).

    Sizes are log-uniform: floor(min_size * (max_size/min_size)^U), clamped.
    Each set is uniform-square, uniform-disk or standard-Gaussian (1/3 each).
    """
    rng = _rng(CONFIG_IDS["batched"], seed)
    ratio = max_size / min_size
    sizes = np.floor(min_size * ratio ** rng.random(num_sets)).astype(np.int64)
    sizes = np.clip(sizes, min_size, max_size)
    kinds = rng.integers(0, 3, size=num_sets)
    offsets = np.zeros(num_sets + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    pts = np.empty((int(offsets[-1]), 2), dtype=np.float32)
    for i in range(num_sets):
        a, b = int(offsets[i]), int(offsets[i + 1])
        m = b - a
        if kinds[i] == 0:
            pts[a:b] = rng.random((m, 2), dtype=np.float32)
        elif kinds[i] == 1:
            pts[a:b] = _disk(rng, m)
        else:
            pts[a:b] = rng.standard_normal((m, 2)).astype(np.float32)
    return pts, offsets


def parabola(n: int = FULL_SIZES["parabola"], seed: int = 0, power: int = 100) -> np.ndarray:
    """Deep-recursion stress: x = fl32(U^power), y = fl32(x^2) as float32[n, 2]."""
    rng = _rng(CONFIG_IDS["parabola"], seed)
    x = (rng.random(n) ** power).astype(np.float32)
    y = (x.astype(np.float64) ** 2).astype(np.float32)
    return np.stack([x, y], axis=1)


def make(name: str, n: int | None = None, seed: int = 0):
    """Generate a workload by name; ``n`` overrides the default size (sets for ``batched``)."""
    fn = {"square": square, "disk": disk, "circle": circle, "degenerate": degenerate,
          "batched": batched, "parabola": parabola}[name]
    if n is None:
        return fn(seed=seed)
    return fn(n, seed=seed)
