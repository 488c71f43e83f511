"""The expected-value study of Sec. 4.2 on a body with a closed form: the
rotated cube [-1, 1]^n with H = {x_1 <= -0.8} cup {x_1 >= 0.8}, so that
E[f] = vol(S cap H) / vol(S) = 0.2 exactly (x_1 is uniform on [-1, 1]).
Every walk, once mixed, must reproduce it within the Monte Carlo error of
its M N points; the indicator kernel must agree with its plain definition
on the chains' points."""
import math

import numpy as np
import pytest

from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


def test_indicator_kernel_matches_definition(spectra):
    n = 6
    A = W.rotated_cube(n, seed=W.BASE_SEED + 70)
    spec = spectra.Spectrahedron(A)
    ch = spectra.Chains(spec, 1000, seed=3)
    ch.hnr(5)
    X = ch.state()[0].cpu().numpy()
    c = W.random_directions(n, 1, seed=4)[0]
    fr = ch.halfspace_fraction(c, -0.3, 0.4, groups=10)
    y = X @ c
    ref = ((y <= -0.3) | (y >= 0.4)).reshape(10, 100).mean(axis=1)
    assert np.array_equal(fr, ref)


def test_study_on_the_cube_is_unbiased_once_mixed(spectra):
    from paper_2010_03817_gb300 import expectation as E
    n = 10
    A = W.rotated_cube(n, seed=W.BASE_SEED + 71)
    spec = spectra.Spectrahedron(A)
    c = np.zeros(n)
    c[0] = 1.0
    res = E.study(spec, c, -0.8, 0.8, lengths=(1, 5, 50), trials=20, points=200,
                  tau=2 * math.sqrt(n), truth=0.2)
    se = E.binomial_se(0.2, 20 * 200)
    for w, rows in res.items():
        last = rows[-1]
        assert last["length"] == 50
        assert last["abs_err"] < 4.5 * se, (w, last)
        # the trials' spread is the binomial spread of N points once mixed
        assert 0.4 * E.binomial_se(0.2, 200) < last["std"] < 2.5 * E.binomial_se(0.2, 200), w
    # one step from the centre (x_1 = 0, inside the slab): CDHR moves x_1 only
    # when it picks coordinate 1 (E = 0.1 * 0.2), Hit-and-Run's chord through
    # the centre rarely reaches |x_1| >= 0.8 -- neither has mixed yet
    assert res["cdhr"][0]["mean"] < 0.1, res["cdhr"][0]
    assert res["hnr"][0]["mean"] < 0.15, res["hnr"][0]
