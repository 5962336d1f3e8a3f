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


def site_rel_max(a, b, site_axes=2):
    """Largest per-site error max_s ||a_s - b_s|| over the RMS per-site norm of b (the trailing
    `site_axes` axes hold one site's components).  An error confined to a few sites (a block face,
    the time boundary) that a whole-field norm would average away shows up here at full size."""
    import numpy as np
    d = np.abs(np.asarray(a) - np.asarray(b)) ** 2
    n = np.abs(np.asarray(b)) ** 2
    ax = tuple(range(d.ndim - site_axes, d.ndim))
    ds = np.sqrt(d.sum(axis=ax))
    rms = np.sqrt(n.sum(axis=ax).mean())
    return float(ds.max() / rms) if rms > 0 else float(ds.max())
