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


@pytest.fixture(scope="session")
def ndf_mod():
    """The ctypes binding over a freshly built libndf.so (GPU tests only)."""
    from paper_2307_02203_gb300 import build

    build.build()
    from paper_2307_02203_gb300 import ndf

    return ndf


@pytest.fixture(scope="session")
def ctx(ndf_mod):
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    c = ndf_mod.ndf_create(0, None)
    yield c
    ndf_mod.ndf_destroy(c)
