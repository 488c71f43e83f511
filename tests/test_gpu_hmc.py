"""Parity of the HMC boundary oracle and walk for the Boltzmann density
exp(-c.x / T) (Sec. 3.3, Alg. 6; the degree-2 trajectory of Sec. 2.1) with
the oracle's reference (oracle/hmc.py: numpy's eigenvalues of the companion
matrix, a dense null vector), plus what the geometry fixes without the
oracle:

* REFLECTION on random lines of S-n-m bodies up to the m = 64 limit, a
  ragged count, more lines than CTAs (t+ to 1e-9 relative, the normal and
  the reflected velocity to 1e-7);
* c = 0: the trajectory is the line and every output equals the GPU's own
  line REFLECTION (sp_reflect, a different solver);
* the rotated cube [-1, 1]^n: t+ is the first root of the per-face scalar
  quadratics, the normal the face's inward unit vector;
* the walk: the first steps of every chain equal the oracle's walk of the
  same chains (same Philox draws), and a long walk on the cube reproduces
  the marginal means of the truncated exponential, E[x_i] = 1/l - coth(l),
  l = c_i / T, within five standard errors.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import hmc
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


def _interior(A, count, scale, seed):
    X = W.random_interior_points(A, 4 * count, scale, seed)
    X = np.array([x for x in X if oracle.membership(A, x)])[:count]
    assert len(X) == count
    return X


def _check_against_oracle(spec, A, X, V, c, T):
    dev = "cuda"
    tp, wh, s, st = spec.curve_reflect(torch.tensor(X, device=dev), torch.tensor(V, device=dev),
                                       c, T)
    tp, wh, s, st = (a.cpu().numpy() for a in (tp, wh, s, st))
    for k in range(len(X)):
        r = hmc.curve_reflect(A, X[k], V[k], c, T)
        assert st[k] == r["status"], k
        if r["status"] != hmc.OK:
            continue
        assert abs(tp[k] - r["t_plus"]) <= 1e-9 * r["t_plus"], (k, tp[k], r["t_plus"])
        assert np.abs(wh[k] - r["w_hat"]).max() <= 1e-7, k
        assert np.abs(s[k] - r["s"]).max() <= 1e-7 * max(1.0, np.abs(r["s"]).max()), k


@pytest.mark.parametrize("n,m,count,T", [(6, 8, 37, 0.5), (20, 20, 200, 2.0), (12, 64, 24, 1.0)])
def test_curve_reflect_matches_oracle(S, n, m, count, T):
    A = W.dabbene(n, m, seed=W.BASE_SEED + 90 + m)
    spec = S.Spectrahedron(A)
    X = _interior(A, count, 0.05, seed=W.BASE_SEED + 91)
    g = np.random.default_rng(92 + m)
    V = g.normal(size=(count, n)) * 0.2
    c = g.normal(size=n)
    _check_against_oracle(spec, A, X, V, c, T)


def test_curve_reflect_ball_random_matches_oracle(S):
    A = W.ball_random(10, 10, 2.0, seed=W.BASE_SEED + 93)
    spec = S.Spectrahedron(A)
    X = _interior(A, 64, 0.5, seed=W.BASE_SEED + 94)
    g = np.random.default_rng(95)
    _check_against_oracle(spec, A, X, g.normal(size=(64, 10)), g.normal(size=10) * 3.0, 0.7)


def test_zero_field_equals_line_reflection(S):
    A = W.dabbene(10, 16, seed=W.BASE_SEED + 96)
    spec = S.Spectrahedron(A)
    X = torch.tensor(_interior(A, 50, 0.05, seed=W.BASE_SEED + 97), device="cuda")
    V = torch.tensor(W.random_directions(10, 50, seed=W.BASE_SEED + 98), device="cuda")
    tp, wh, s, st = spec.curve_reflect(X, V, np.zeros(10), 1.0)
    tl, whl, sl, stl = spec.reflect(X, V)
    assert (st == 0).all() and (stl == 0).all()
    assert torch.allclose(tp, tl, rtol=1e-10, atol=0)
    assert (wh - whl).abs().max().item() <= 1e-8
    assert (s - sl).abs().max().item() <= 1e-8


def _first_root_cube(p, v, c, T):
    best, face = np.inf, None
    a2 = -c / (2 * T)
    for i in range(len(p)):
        for sgn in (1.0, -1.0):
            r = np.roots([a2[i], v[i], p[i] - sgn])
            for t in np.atleast_1d(r):
                if np.imag(t) == 0 and np.real(t) > 1e-14 and np.real(t) < best:
                    best, face = float(np.real(t)), (i, sgn)
    return best, face


def test_cube_closed_form(S):
    n, T = 5, 0.8
    A = W.rotated_cube(n, seed=W.BASE_SEED + 99)
    spec = S.Spectrahedron(A)
    g = np.random.default_rng(100)
    P = g.uniform(-0.9, 0.9, size=(40, n))
    V = g.normal(size=(40, n))
    c = g.normal(size=n)
    c[c == 0] = 0.1
    tp, wh, s, st = spec.curve_reflect(torch.tensor(P, device="cuda"),
                                       torch.tensor(V, device="cuda"), c, T)
    tp, wh, s = (a.cpu().numpy() for a in (tp, wh, s))
    assert (st == 0).all()
    for k in range(40):
        t_ref, (i, sgn) = _first_root_cube(P[k], V[k], c, T)
        assert abs(tp[k] - t_ref) <= 1e-10 * t_ref
        e = np.zeros(n)
        e[i] = -sgn
        assert np.abs(wh[k] - e).max() <= 1e-8
        vel = V[k] - c / T * t_ref
        vel[i] = -vel[i]
        assert np.abs(s[k] - vel).max() <= 1e-8 * max(1.0, np.abs(vel).max())


def test_status_and_errors(S):
    A = W.dabbene(6, 8, seed=W.BASE_SEED + 101)
    spec = S.Spectrahedron(A)
    x = torch.full((2, 6), 50.0, dtype=torch.float64, device="cuda")  # far outside
    x[1] = 0.0
    v = torch.ones((2, 6), dtype=torch.float64, device="cuda")
    tp, wh, s, st = spec.curve_reflect(x, v, np.ones(6), 1.0)
    assert st.tolist()[0] == 1 and st.tolist()[1] == 0  # SP_ST_NOTPD, then OK
    assert (wh[0] == 0).all()
    with pytest.raises(S.SpectraError):
        spec.curve_reflect(x, v, np.ones(6), 0.0)
    big = S.Spectrahedron(W.dabbene(4, 66, seed=W.BASE_SEED + 102))
    with pytest.raises(S.SpectraError):
        big.curve_reflect(torch.zeros((1, 4), dtype=torch.float64, device="cuda"),
                          torch.ones((1, 4), dtype=torch.float64, device="cuda"), np.ones(4), 1.0)


def test_walk_matches_the_oracle_walk(S):
    n, m, T, tau, seed = 8, 12, 1.0, 1.0, 77
    A = W.dabbene(n, m, seed=W.BASE_SEED + 103)
    spec = S.Spectrahedron(A)
    C, steps = 48, 3
    X0 = _interior(A, C, 0.02, seed=W.BASE_SEED + 104)
    c = np.random.default_rng(105).normal(size=n)
    ch = S.Chains(spec, C, x0=X0, seed=seed)
    ch.hmc(steps, c, T, tau, rho=100, kappa=1e-6)
    Xg, step = ch.state_host()
    assert step == steps
    for k in range(C):
        x = X0[k].copy()
        for j in range(steps):
            x, st, _ = hmc.hmc_step(A, x, c, T, tau=tau, rho=100, kappa=1e-6, seed=seed,
                                    chain=k, step=j)
            assert st == 0
        assert np.abs(Xg[k] - x).max() <= 1e-8 * max(1.0, np.abs(x).max()), k


def test_boltzmann_cube_marginals(S):
    n, T = 4, 1.0
    c = np.array([2.0, -1.0, 0.5, 0.0])
    A = W.rotated_cube(n, seed=W.BASE_SEED + 106)
    spec = S.Spectrahedron(A)
    C = 4096
    ch = S.Chains(spec, C, seed=11)
    ch.hmc(40, c, T, tau=2.0, rho=1000, kappa=1e-6)
    X, _ = ch.state_host()
    assert np.abs(X).max() < 1.0
    for i in range(n):
        lam = c[i] / T
        if lam == 0:
            mean, var = 0.0, 1.0 / 3.0
        else:
            mean = 1.0 / lam - 1.0 / math.tanh(lam)
            var = 1.0 / lam ** 2 - 1.0 / math.sinh(lam) ** 2
        se = math.sqrt(var / C)
        assert abs(X[:, i].mean() - mean) <= 5 * se, (i, X[:, i].mean(), mean, se)


def test_fig4_boltzmann_means(S, example_2d):
    """Fig. 4 (right): T = 1, c = (-0.09, 1) on the Appendix B spectrahedron;
    4096 GPU chains from (-1, 1) reproduce the density's mean (quadrature)
    within five standard errors."""
    import conftest
    A = example_2d
    c, T = np.array([-0.09, 1.0]), 1.0
    mean, var, _ = conftest.boltzmann_moments_2d(A, c, T)
    spec = S.Spectrahedron(A)
    C = 4096
    ch = S.Chains(spec, C, x0=np.tile([-1.0, 1.0], (C, 1)), seed=23)
    ch.hmc(25, c, T, tau=6.0, rho=100, kappa=1e-6)
    X, _ = ch.state_host()
    _, stats = ch.status()
    assert stats["bad_steps"] == 0 and stats["reflections"] > 0
    se = np.sqrt(var / C)
    assert np.all(np.abs(X.mean(axis=0) - mean) <= 5 * se), (X.mean(axis=0), mean, se)
