import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session", autouse=True)
def _host_builds():
    """Build the CPU oracle and the input generators once per session."""
    import oracle
    import synth

    oracle.build()
    if not (os.path.exists(synth.HOST_LIB) and os.path.exists(synth.CUDA_LIB)):
        synth.build()
    yield


def gpu_available() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def mwax_lib():
    """The CUDA library, built for sm_103a (built here if missing)."""
    import paper_0902_0915_gb300 as mw

    mw.ensure_built()
    return mw
