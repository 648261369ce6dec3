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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_count(name):
    """A count the paper states about its grids (tests/golden/paper_counts.txt)."""
    with open(os.path.join(GOLDEN, "paper_counts.txt")) as fh:
        for line in fh:
            f = line.split()
            if f and not f[0].startswith("#") and f[0] == name:
                return int(f[1])
    raise KeyError(name)


def control_cube_tets():
    """The paper's 24 control-cube tetrahedra (tests/golden/control_cube_24_tets.txt): a list
    of frozensets of 4 points, in units of half the cube edge."""
    out = []
    with open(os.path.join(GOLDEN, "control_cube_24_tets.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = [int(x) for x in line.split()]
                out.append(frozenset(tuple(v[3 * k:3 * k + 3]) for k in range(4)))
    return out
