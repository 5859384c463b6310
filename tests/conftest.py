import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")
    config.addinivalue_line(
        "markers",
        "gpu_pending: GPU test of code that has not yet run on a GB300; kept out of -m gpu until it has "
        "passed there once (run it with -m gpu_pending); skips without a CUDA device")
