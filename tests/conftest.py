import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libtdmrg.so")


@pytest.fixture(scope="session")
def c1_problem():
    """L=8 Hubbard chain, t=1, U=4, 4 up + 4 down: both halves exact (m = 256)."""
    from oracle import models
    return models.chain(8, t=1.0, U=4.0)


@pytest.fixture(scope="session")
def c1_ground(c1_problem):
    return c1_problem.ground_state()
