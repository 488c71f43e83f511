import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")


def load_example_2d():
    """The Appendix B matrices (tests/golden/example_2d.txt) as a (3, 6, 6) stack."""
    path = os.path.join(ROOT, "tests", "golden", "example_2d.txt")
    mats, cur = [], None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("A"):
            cur = []
            mats.append(cur)
            continue
        cur.append([float(t) for t in line.split()])
    return np.array(mats, dtype=np.float64)


@pytest.fixture(scope="session")
def example_2d():
    return load_example_2d()
