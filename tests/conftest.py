import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def tiny_set():
    from synth import configs
    return configs.tiny_set()


@pytest.fixture(scope="session")
def tiny_set_holes():
    from synth import configs
    return configs.tiny_set(seed=11, n_blocks=400, holes=0.1)


@pytest.fixture(scope="session")
def state_set():
    """The state-scale set (199,972 blocks); about 20 s to generate."""
    from synth import configs
    return configs.state_set()
