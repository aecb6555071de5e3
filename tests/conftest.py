import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def tiny_band():
    import synth
    return synth.make_band(synth.CONFIGS["tiny"])


@pytest.fixture(scope="session")
def tiny_ingest(tiny_band):
    import oracle
    return oracle.ingest(tiny_band)
