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
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libndf.so")
    config.addinivalue_line("markers", "slow: longer CPU statistical checks")


@pytest.fixture(scope="session")
def tiny_field():
    import synth

    return synth.generate(synth.TINY)


@pytest.fixture(scope="session")
def tiny_ref():
    import synth

    x, y, z = synth.TINY_REF
    return synth.vertex_index(x, y, z, synth.TINY)
