"""Planted mistakes in the oracle (built on the CPU) must be caught by the pins.

Each variant of qh_oracle.c is compiled with -DQHO_MUTATION=k:
  1  keeps collinear boundary points (pop only on a strict right turn)
  2  flips the sign of one product in orient
  3  keeps the highest index among duplicate coordinates
  4  sorts ties in x by descending y
  5  trusts any non-zero double sum (no error bound)
  6  breaks farthest-point ties by the higher index
"""
import pytest

import pins


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5, 6])
def test_mutation_is_caught(mutation):
    failed = pins.run_all(mutation)
    assert failed, f"mutation {mutation} passed every pin"
