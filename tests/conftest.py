import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built librogs")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_runtest_setup(item):
    """A GPU test on a machine without a CUDA device fails when GPU tests were
    asked for explicitly (-m gpu), so that such a run cannot pass by skipping
    everything; in an unfiltered run it is skipped."""
    if item.get_closest_marker("gpu") is None or _cuda_available():
        return
    if item.config.getoption("-m", default="").strip() == "gpu":
        pytest.fail("GPU test selected with -m gpu, but no CUDA device is available", pytrace=False)
    pytest.skip("no CUDA device")
