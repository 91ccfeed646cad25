import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: full-size cases (still run by -m gpu)")


@pytest.fixture(scope="session")
def gpu():
    """The CUDA binding; GPU tests fail loudly when the extension is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a -m gpu test ran without a visible CUDA device")
    import paper_1702_07961_gb300 as mms
    mms.load()  # raises if libmms.so is missing: no fallback exists
    return mms
