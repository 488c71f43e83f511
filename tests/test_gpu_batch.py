"""A batch of spectrahedra of uneven sizes in one persistent launch.

* With the default panel width, every chain of the batch walks exactly as the
  same chain walked alone through sp_step_billiard (the same Philox stream,
  chain0 = the body's offset, and the same arithmetic): bitwise equal.
* With the tuned panel widths, the same to rounding.
* The first step of sampled chains of every body follows the oracle's walk.
* The tuner writes its cache and a second tuning reads it back.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(8, 12), (15, 6), (5, 30), (20, 20)]  # (n, k): m = n + 1 + k
CHAINS = [24, 40, 16, 32]
SEED = 5
TAU = 6.0  # 2 r for the ball block r = 3


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


@pytest.fixture(scope="module")
def bodies():
    return [W.ball_random(n, k, 3.0, seed=W.BASE_SEED + 200 + i)
            for i, (n, k) in enumerate(SIZES)]


def _alone(spectra, A, C, chain0, steps):
    spec = spectra.Spectrahedron(A)
    ch = spectra.Chains(spec, C, seed=SEED, chain0=chain0)
    ch.billiard(steps, tau=TAU, rho=100, kappa=1e-6)
    return ch.state()[0].cpu().numpy()


def test_batch_equals_single_body_walks(spectra, bodies):
    specs = [spectra.Spectrahedron(A) for A in bodies]
    b = spectra.Batch(specs, CHAINS, seed=SEED)
    assert list(b.panels()) == [8, 8, 8, 8]
    b.billiard(2, TAU)
    for i, A in enumerate(bodies):
        n, m, c, c0 = b.dims(i)
        assert (n, m, c) == (SIZES[i][0], SIZES[i][0] + 1 + SIZES[i][1], CHAINS[i])
        assert c0 == sum(CHAINS[:i])
        xb = b.state(i)
        xa = _alone(spectra, A, CHAINS[i], c0, 2)
        assert np.array_equal(xb, xa), (i, np.abs(xb - xa).max())
    st = b.stats()
    for i in range(len(bodies)):
        assert st[i]["segments"] >= 2 * CHAINS[i]
        assert st[i]["bad_steps"] == 0


def test_batch_with_tuned_panels(spectra, bodies, tmp_path):
    specs = [spectra.Spectrahedron(A) for A in bodies]
    b = spectra.Batch(specs, CHAINS, seed=SEED)
    cache = str(tmp_path / "panels.tsv")
    panels, times = b.tune(cache)
    assert set(panels.tolist()) <= {4, 8, 16}
    assert (times > 0).all()
    assert os.path.exists(cache)
    lines = [ln for ln in open(cache) if not ln.startswith("#")]
    assert len(lines) == len(bodies)
    # the cache answers a second tuning (the same widths and times)
    b2 = spectra.Batch(specs, CHAINS, seed=SEED)
    panels2, times2 = b2.tune(cache)
    assert np.array_equal(panels, panels2)
    assert np.allclose(times, times2, rtol=1e-6, atol=0.0)
    # every width gives the same walk to rounding
    b.panels([16, 4, 16, 4])
    b.billiard(1, TAU)
    b2.panels([4, 16, 8, 16])
    b2.billiard(1, TAU)
    for i in range(len(bodies)):
        d = np.abs(b.state(i) - b2.state(i))
        assert np.median(d) < 1e-12 and d.max() < 1e-8, (i, d.max())


def test_batch_first_step_follows_oracle(spectra, bodies):
    specs = [spectra.Spectrahedron(A) for A in bodies]
    b = spectra.Batch(specs, CHAINS, seed=SEED)
    b.billiard(1, TAU)
    for i, A in enumerate(bodies):
        n, _, c, c0 = b.dims(i)
        xb = b.state(i)
        k = 6
        Xo, _ = oracle.walk("billiard", A, np.zeros((k, n)), 1, tau=TAU, rho=100, kappa=1e-6,
                            seed=SEED, step0=0, chain0=c0)
        assert np.abs(xb[:k] - Xo).max() < 1e-9, i


def test_batch_rejects_bad_arguments(spectra, bodies):
    specs = [spectra.Spectrahedron(A) for A in bodies[:2]]
    with pytest.raises(spectra.SpectraError):
        spectra.Batch(specs, [4, 0])
    b = spectra.Batch(specs, [4, 4])
    with pytest.raises(spectra.SpectraError):
        b.panels([8, 5])
    with pytest.raises(spectra.SpectraError):
        b.billiard(1, [1.0, -1.0])
