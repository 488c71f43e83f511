"""GPU walks (Alg. 4 Hit-and-Run, CDHR, Alg. 5 Billiard) against the oracle:
per-step agreement on the same Philox streams while trajectories are still
close, moments within Monte-Carlo error, the invariant F(x) > 0 for every
emitted point, and parity of the boundary oracle on states a Billiard walk
actually visits (points kappa-close to the boundary after a reflection)."""
import math

import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


def test_first_steps_follow_oracle(spectra):
    """Config-1 construction (n = 10, ball r = 3 + random block k = 10, m = 21):
    same seed, same counters -> the same first step (to rounding; CUDA's and
    the host's log/sin/cos may differ in the last ulp), and after three steps
    most chains still agree closely (reflections amplify differences)."""
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED + 0)
    spec = spectra.Spectrahedron(A)
    for kind in ["billiard", "hnr", "cdhr"]:
        ch = spectra.Chains(spec, 32, seed=11)
        Xo = np.zeros((32, n))
        for k in range(3):
            if kind == "billiard":
                ch.billiard(1, tau=6.0, rho=100, kappa=1e-6)
            else:
                getattr(ch, kind)(1)
            Xo, so = oracle.walk(kind, A, Xo, 1, tau=6.0, rho=100, kappa=1e-6, seed=11, step0=k)
            xs, step = ch.state()
            assert step == k + 1
            err = np.abs(xs.cpu().numpy() - Xo).max(axis=1)
            if k == 0:
                assert err.max() < 1e-9, kind
        assert np.median(err) < 1e-9 and np.mean(err < 1e-6) > 0.8, kind


@pytest.mark.parametrize("kind", ["billiard", "hnr", "cdhr"])
def test_cube_marginals(spectra, kind):
    n, C = 5, 2048
    A = W.rotated_cube(n, seed=W.BASE_SEED + 1)
    spec = spectra.Spectrahedron(A)
    ch = spectra.Chains(spec, C, seed=21)
    if kind == "billiard":
        ch.billiard(20, tau=2 * math.sqrt(n), rho=100, kappa=1e-6)
    else:
        getattr(ch, kind)(40)
    X = ch.state()[0].cpu().numpy()
    st, stats = ch.status()
    assert stats["bad_steps"] == 0, (stats, np.unique(st.cpu().numpy(), return_counts=True))
    se_mean = math.sqrt(1.0 / 3.0 / C)
    se_var = math.sqrt((1.0 / 5.0 - 1.0 / 9.0) / C)
    assert np.all(np.abs(X.mean(0)) < 4.5 * se_mean)
    assert np.all(np.abs((X ** 2).mean(0) - 1.0 / 3.0) < 4.5 * se_var)
    assert np.all(np.abs(X) < 1.0)


def test_ball_second_moment_and_invariant(spectra):
    n, C, R = 8, 2048, 1.0
    A = W.ball(n, R)
    spec = spectra.Spectrahedron(A)
    ch = spectra.Chains(spec, C, seed=22)
    ch.billiard(25, tau=2 * R, rho=100, kappa=1e-6)
    x, _ = ch.state()
    assert bool(spec.membership(x).all())
    X = x.cpu().numpy()
    r2 = (X ** 2).sum(1)
    expect = n * R * R / (n + 2)
    var = n * R ** 4 / (n + 4) - expect ** 2
    assert abs(r2.mean() - expect) < 4.5 * math.sqrt(var / C)


def test_config1_walks_match_oracle_in_distribution(spectra):
    """64 chains x 1000 steps from x = 0 (Billiard and Hit-and-Run, FP64):
    every point interior; chain-mean of x and |x|^2 agree with the oracle's
    own run within Monte-Carlo error."""
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED + 0)
    spec = spectra.Spectrahedron(A)
    for kind in ["billiard", "hnr"]:
        ch = spectra.Chains(spec, 64, seed=31)
        samples = []
        for _ in range(10):
            if kind == "billiard":
                ch.billiard(100, tau=6.0, rho=100, kappa=1e-6)
            else:
                ch.hnr(100)
            x, _ = ch.state()
            assert bool(spec.membership(x).all())
            samples.append(x.cpu().numpy())
        G = np.concatenate(samples[2:])
        Xo = np.zeros((64, n))
        osamp = []
        for b in range(10):
            Xo, _ = oracle.walk(kind, A, Xo, 100, tau=6.0, rho=100, kappa=1e-6, seed=32,
                                step0=100 * b)
            osamp.append(Xo.copy())
        O = np.concatenate(osamp[2:])
        for fg, fo in [(G, O), ((G ** 2).sum(1, keepdims=True), (O ** 2).sum(1, keepdims=True))]:
            se = np.sqrt(fg.var(0) / len(fg) * 4 + fo.var(0) / len(fo) * 4)  # autocorrelation slack
            assert np.all(np.abs(fg.mean(0) - fo.mean(0)) < 5 * se + 1e-12), kind


def _billiard_states(A, x0, tau, seed, chain, steps):
    """(p, v) at every segment of a few oracle Billiard steps (the same rules
    as Alg. 5 with kappa = 1e-6), for parity on visited states."""
    n = A.shape[0] - 1
    out = []
    x = x0.copy()
    for st in range(steps):
        v = oracle.direction(n, seed, chain, st)
        ell = -tau * math.log(oracle.uniform(seed, chain, st, 1))
        p = x.copy()
        for _ in range(50):
            out.append((p.copy(), v.copy()))
            r = oracle.reflect(A, p, v)
            if r["t_plus"] < ell:
                p = p + (1 - 1e-6) * r["t_plus"] * v
                ell -= r["t_plus"]
                v = r["s"]
            else:
                x = p + ell * v
                break
    return out


def test_parity_on_post_reflection_states(spectra):
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED + 0)
    states = _billiard_states(A, np.zeros(n), 12.0, 41, 0, 6)
    X = np.array([s[0] for s in states])
    V = np.array([s[1] for s in states])
    assert len(states) > 10
    spec = spectra.Spectrahedron(A)
    tp, wh, s, st = spec.reflect(torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda"))
    tp, wh = tp.cpu().numpy(), wh.cpu().numpy()
    for c in range(len(X)):
        rf = oracle.reflect(A, X[c], V[c])
        assert abs(tp[c] - rf["t_plus"]) <= 1e-10 * rf["t_plus"], c
        if rf["rel_gap"] > 1e-6:
            assert np.abs(wh[c] - rf["w_hat"]).max() <= 1e-9, c


def test_rho_zero_keeps_points(spectra):
    n = 4
    A = W.rotated_cube(n, seed=3)
    spec = spectra.Spectrahedron(A)
    x0 = np.full((64, n), 0.1)
    ch = spectra.Chains(spec, 64, x0=x0, seed=5)
    ch.billiard(1, tau=100.0, rho=0, kappa=1e-6)
    X = ch.state()[0].cpu().numpy()
    st, stats = ch.status()
    moved = np.any(X != x0, axis=1)
    # tau = 100 on a cube of diameter 4: (almost) every step reflects and is rejected
    assert stats["bad_steps"] == int((~moved).sum()) > 0
    assert np.all(st.cpu().numpy()[~moved] == spectra.ST_RHO)


def test_checkpoint_resume_is_exact(spectra):
    n = 6
    A = W.ball_random(n, 6, 2.0, seed=7)
    spec = spectra.Spectrahedron(A)
    a = spectra.Chains(spec, 16, seed=9)
    a.billiard(8, tau=4.0)
    b = spectra.Chains(spec, 16, seed=9)
    b.billiard(4, tau=4.0)
    xh, step = b.state_host()
    c = spectra.Chains(spec, 16, seed=9)
    c.set_state(xh, step)
    c.billiard(4, tau=4.0)
    assert np.array_equal(a.state_host()[0], c.state_host()[0])
