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


def boltzmann_moments_2d(A, c, T, half=7.0, k=561):
    """E[x] and Var[x] of exp(-c.x / T) restricted to the 2D spectrahedron,
    by the midpoint rule on a k x k grid over [-half, half]^2 (membership by
    numpy's eigenvalues of F(x); the body must not touch the grid's border)."""
    h = 2 * half / k
    g = -half + h * (np.arange(k) + 0.5)
    X1, X2 = np.meshgrid(g, g, indexing="ij")
    F = A[0][None, None] + X1[..., None, None] * A[1] + X2[..., None, None] * A[2]
    inside = np.linalg.eigvalsh(F)[..., 0] > 0
    assert not inside[0].any() and not inside[-1].any()
    assert not inside[:, 0].any() and not inside[:, -1].any()
    wgt = np.where(inside, np.exp(-(c[0] * X1 + c[1] * X2) / T), 0.0)
    Z = wgt.sum()
    mean = np.array([(wgt * X1).sum(), (wgt * X2).sum()]) / Z
    var = np.array([(wgt * X1 ** 2).sum(), (wgt * X2 ** 2).sum()]) / Z - mean ** 2
    return mean, var, inside.sum() * h * h


@pytest.fixture(scope="session")
def example_2d():
    return load_example_2d()
