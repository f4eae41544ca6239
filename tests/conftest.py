import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs through the C-ABI library)")
    config.addinivalue_line("markers", "slow: full-size workloads")


@pytest.fixture(scope="session")
def qh():
    """The product binding, loaded once; skips when no GPU is visible."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_04706_gb300 as qh_mod

    qh_mod.load()
    return qh_mod
