"""Pins for the CPU oracle: each check compares it with something other than itself."""
import numpy as np
import pytest

import oracle
import pins


def test_orient_exact_vs_rationals():
    pins.check_orient()


def test_dist_cmp_exact_vs_rationals():
    pins.check_dist_cmp()


def test_golden_fixtures():
    assert len(pins.golden_cases()) >= 8
    pins.check_golden()


def test_brute_force_small_random():
    pins.check_brute_random()


def test_every_subset_of_3x3_grid():
    pins.check_grid_subsets()


def test_closed_forms():
    pins.check_closed_forms()


def test_invariants_medium_workloads():
    pins.check_invariants_medium()


def test_metamorphic_relations():
    pins.check_metamorphic()


def test_batched_equals_per_set():
    pins.check_batched()


def test_nonfinite_rejected():
    p = np.array([[0, 0], [1, np.nan], [2, 2]], dtype=np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.hull2d(p)
    assert e.value.status == oracle.NONFINITE
    p[1, 1] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.quickhull(p)


def test_always_exact_agrees_with_filtered():
    import synth

    p = synth.degenerate(20000, grid=128)
    assert np.array_equal(oracle.hull2d(p), oracle.hull2d(p, always_exact=True))
