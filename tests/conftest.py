import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cfg_small():
    """The plain FP64 CCA workload: n=2000, dx=50, dy=40, k=5, lambda=1e-3."""
    from synth import cca_latent_problem
    return cca_latent_problem(2000, 50, 40, latent=10, noise=0.5, dtype="f64", seed=0)
