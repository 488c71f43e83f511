"""Volume by multiphase Monte Carlo over a sequence of balls (Sec. 4.1),
judged against exact volumes: the cube [-1, 1]^n (2^n, here as the rotated
cube LMI) and the n-ball (pi^(n/2) r^n / Gamma(n/2 + 1)), with the Billiard
and Hit-and-Run samplers.  The tolerance combines the estimator's own
binomial standard error (reported) with the walks' autocorrelation, which
that error ignores: 6 % relative."""
import math

import pytest

from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


@pytest.mark.parametrize("walk", ["billiard", "hnr"])
def test_cube_volume(spectra, walk):
    n = 6
    spec = spectra.Spectrahedron(W.rotated_cube(n, seed=W.BASE_SEED + 4))
    vol, info = spec.volume(1.0, math.sqrt(n), ratio=0.5, chains=4096, burn_in=10, steps=20,
                            walk=walk)
    assert info["phases"] == math.ceil(n * math.log(math.sqrt(n)) / math.log(2.0))
    assert abs(vol / 2.0 ** n - 1.0) < 0.06, (vol, info)


def test_ball_volume(spectra):
    n, r = 8, 1.0
    spec = spectra.Spectrahedron(W.ball(n, r))
    exact = math.pi ** (n / 2) * r ** n / math.gamma(n / 2 + 1)
    vol, info = spec.volume(0.5 * r, r, ratio=0.5, chains=4096, burn_in=10, steps=20)
    assert abs(vol / exact - 1.0) < 0.06, (vol, exact, info)


def test_mixed_mode_agrees(spectra):
    n = 6
    spec = spectra.Spectrahedron(W.rotated_cube(n, seed=W.BASE_SEED + 4))
    vol, _ = spec.volume(1.0, math.sqrt(n), chains=2048, burn_in=10, steps=20, mode="mixed")
    assert abs(vol / 2.0 ** n - 1.0) < 0.08


def test_bad_arguments(spectra):
    spec = spectra.Spectrahedron(W.ball(4, 1.0))
    with pytest.raises(spectra.SpectraError):
        spec.volume(1.0, 0.5)
    with pytest.raises(spectra.SpectraError):
        spec.volume(0.5, 1.0, ratio=1.5)
