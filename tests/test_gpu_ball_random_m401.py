"""The paper's top size with the learned configuration's body: n = 200,
F = blockdiag(ball block r = 3 (m = 201), random block k = 200) (m = 401).
Both GPU paths treat F as dense; the factor (645 KB in FP64) no longer fits
one block's shared memory, so the FP64 path keeps it in global memory and
the mixed path its work region; the normals take the in-kernel contraction
(the tensor-core one stops at m = 224).  Checked against the oracle on lines
its own Billiard walk meets and on the walk's first step."""
import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, K, R = 200, 200, 3.0
TAU = 2 * R
TOL_T = {"fp64": 1e-10, "mixed": 1e-9}


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


@pytest.fixture(scope="module")
def body():
    return W.ball_random(N, K, R, seed=W.BASE_SEED + 4)


@pytest.fixture(scope="module")
def spec(spectra, body):
    return spectra.Spectrahedron(body)


@pytest.fixture(scope="module")
def traced(body):
    """The lines of the oracle's first Billiard step of 8 chains from the
    origin (every line after a chain's first starts kappa-close to the
    boundary)."""
    Xo, P, V, st, rows = oracle.billiard_trace(body, np.zeros((8, N)), 0, tau=TAU, rho=100,
                                               kappa=1e-6, seed=9, max_per_chain=3)
    ref = oracle.reflect_batch(body, P, V)
    keep = ref["status"] == 0
    return P[keep], V[keep], {k: np.asarray(v)[keep] for k, v in ref.items()}, (st, Xo)


def test_dims(body):
    assert body.shape == (N + 1, 401, 401)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_reflect_on_traced_lines(spectra, spec, traced, mode):
    P, V, ref, _ = traced
    assert len(P) >= 10
    tp, wh, s, st = spec.reflect(torch.tensor(P, device="cuda"), torch.tensor(V, device="cuda"),
                                 mode=mode)
    tp, wh, st = tp.cpu().numpy(), wh.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all(), (mode, st)
    et = np.abs(tp - ref["t_plus"]) / ref["t_plus"]
    assert et.max() <= TOL_T[mode], (mode, et.max())
    gap = ref["rel_gap"] > 1e-6
    if gap.any():
        assert np.abs(wh[gap] - ref["w_hat"][gap]).max() <= TOL_T[mode], mode


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_first_step_follows_oracle(spectra, spec, body, traced, mode):
    """Chains 0..7 of a 64-chain walk from the origin, seed 9: their first
    step is the oracle's traced step."""
    _, _, _, (st, Xo) = traced
    assert (st == 0).all()
    ch = spectra.Chains(spec, 64, seed=9)
    ch.billiard(1, tau=TAU, rho=100, kappa=1e-6, mode=mode)
    x = ch.state()[0].cpu().numpy()
    assert np.abs(x[:8] - Xo).max() < 1e-9, mode
    assert bool(spec.membership(torch.tensor(x, device="cuda")).all())
