import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: oracle test that takes more than ~20 s on one core")


def rel(a, b):
    import numpy as np
    d = np.linalg.norm(np.ravel(a - b))
    n = np.linalg.norm(np.ravel(b))
    return d / n if n > 0 else d
