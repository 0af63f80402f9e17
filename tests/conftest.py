import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def geom_full():
    from paper_2403_13166_gb300 import synth
    return synth.build_geometry(True)


@pytest.fixture(scope="session")
def geom_toy():
    from paper_2403_13166_gb300 import synth
    return synth.build_geometry(False)


@pytest.fixture(scope="session")
def cuts():
    from paper_2403_13166_gb300 import synth
    return synth.default_cuts()
