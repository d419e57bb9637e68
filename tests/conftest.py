import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def cuda_lib():
    """The built CUDA library; on a GPU machine a missing library is a failure, not a skip."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_1708_08640_gb300 import _lib
    return _lib.load(build_if_missing=True)


@pytest.fixture(scope="session")
def rating_tensor():
    """The cfg1 workload (3-way 100000 x 50000 x 1000 rating tensor, 10M entries, coupled
    100000 x 100000 binary matrix), generated once per session."""
    from paper_1708_08640_gb300 import synth
    return synth.make_problem("cfg1")
