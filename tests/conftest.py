import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def golden_path(name):
    return os.path.join(GOLDEN, name)


def golden_lines(name):
    with open(golden_path(name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


@pytest.fixture
def has_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True
