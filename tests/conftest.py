import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU case")


_VOL_CACHE = {}


def scene_volume(name, **kw):
    """Volume of a named scene as a numpy array (generated once per process)."""
    from paper_2506_11510_gb300 import workloads as W
    key = (name, tuple(sorted(kw.items())))
    if key not in _VOL_CACHE:
        s = W.scene(name, **kw)
        _VOL_CACHE[key] = W.make_volume(s).numpy()
    return _VOL_CACHE[key]


@pytest.fixture(scope="session")
def tiny_volume():
    return scene_volume("tiny")
