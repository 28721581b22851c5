import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU run")


def load_patch_nodes():
    """16x3 patch-test coordinates of Fig. 2(c) (tests/golden/patch_nodes.txt)."""
    a = np.loadtxt(os.path.join(GOLDEN, "patch_nodes.txt"), comments="#")
    assert a.shape == (16, 4) and np.all(a[:, 0] == np.arange(1, 17))
    return a[:, 1:]


@pytest.fixture(scope="session")
def patch_nodes():
    return load_patch_nodes()
