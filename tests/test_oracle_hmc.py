"""Pins of the HMC oracle (the degree-2 trajectory of Alg. 6 for the
Boltzmann density) against what the geometry fixes without it:

* c = 0: the trajectory is the line, and every output equals the line
  oracle's REFLECTION (a different code path: Jacobi on the linear pencil).
* The rotated cube [-1, 1]^n: Phi_i(t) = p_i + v_i t - c_i t^2 / (2T) meets a
  face where a scalar quadratic vanishes; the first root over all faces is
  t+, the face normal is -+e_i (pointing inward) and the reflection flips
  the i-th component of the velocity Phi'(t+).
* The ball |x| <= r: |Phi(t)|^2 = r^2 is a quartic in t (library roots); the
  normal at the hit point q is -q/|q|.
* The walk keeps every point inside and follows the trajectory it states.
"""
import numpy as np
import pytest

import conftest
import oracle
from oracle import hmc
from paper_2010_03817_gb300 import workloads as W


def _first_root_cube(p, v, c, T):
    best, face = np.inf, None
    a2 = -c / (2 * T)
    for i in range(len(p)):
        for sgn in (1.0, -1.0):
            # p_i + v_i t + a2_i t^2 = sgn
            r = np.roots([a2[i], v[i], p[i] - sgn]) if a2[i] != 0 else np.array(
                [(sgn - p[i]) / v[i]] if v[i] != 0 else [])
            for t in np.atleast_1d(r):
                if abs(np.imag(t)) == 0 and np.real(t) > 1e-14 and np.real(t) < best:
                    best, face = float(np.real(t)), (i, sgn)
    return best, face


def test_line_limit_equals_the_line_oracle():
    A = W.ball_random(5, 4, 2.0, seed=W.BASE_SEED + 80)
    g = np.random.default_rng(1)
    for _ in range(4):
        p = g.uniform(-0.2, 0.2, 5)
        v = W.random_directions(5, 1, seed=int(g.integers(1 << 30)))[0]
        r = hmc.curve_reflect(A, p, v, np.zeros(5), 1.0)
        ro = oracle.reflect(A, p, v)
        assert r["status"] == 0 and ro["status"] == 0
        assert abs(r["t_plus"] - ro["t_plus"]) <= 1e-12 * ro["t_plus"]
        assert np.allclose(r["w_hat"], ro["w_hat"], atol=1e-10)
        assert np.allclose(r["s"], ro["s"], atol=1e-10)


@pytest.mark.parametrize("T", [0.3, 1.0, 5.0])
def test_cube_closed_form(T):
    n = 4
    A = W.rotated_cube(n, seed=W.BASE_SEED + 81)
    g = np.random.default_rng(2)
    for _ in range(6):
        p = g.uniform(-0.8, 0.8, n)
        v = g.normal(size=n)
        c = g.normal(size=n)
        t_ref, (i, sgn) = _first_root_cube(p, v, c, T)
        roots = hmc.curve_roots(A, p, v, c, T)
        assert abs(roots[0] - t_ref) <= 1e-9 * t_ref
        r = hmc.curve_reflect(A, p, v, c, T)
        assert abs(r["t_plus"] - t_ref) <= 1e-12 * t_ref
        e = np.zeros(n)
        e[i] = -sgn
        assert np.allclose(r["w_hat"], e, atol=1e-9)
        vel = v - c / T * t_ref
        s_ref = vel.copy()
        s_ref[i] = -vel[i]
        assert np.allclose(r["s"], s_ref, atol=1e-9)


def test_ball_quartic():
    n, R, T = 5, 1.5, 0.7
    A = W.ball(n, R)
    g = np.random.default_rng(3)
    for _ in range(6):
        p = g.uniform(-0.4, 0.4, n)
        v = g.normal(size=n)
        c = g.normal(size=n) * 2.0
        a = -c / (2 * T)
        coef = [a @ a, 2 * (v @ a), v @ v + 2 * (p @ a), 2 * (p @ v), p @ p - R * R]
        rr = np.roots(coef)
        t_ref = min(float(np.real(t)) for t in rr if abs(np.imag(t)) < 1e-12 and np.real(t) > 0)
        r = hmc.curve_reflect(A, p, v, c, T)
        assert abs(r["t_plus"] - t_ref) <= 1e-10 * t_ref
        q = p + v * t_ref + a * t_ref ** 2
        assert np.allclose(r["w_hat"], -q / np.linalg.norm(q), atol=1e-8)


def test_hmc_step_stays_inside_and_moves_on_the_parabola():
    n = 3
    A = W.rotated_cube(n, seed=W.BASE_SEED + 82)
    c = np.array([1.0, -0.5, 0.3])
    x = np.zeros(n)
    for k in range(20):
        x_new, st, refl = hmc.hmc_step(A, x, c, 1.0, tau=3.0, rho=100, kappa=1e-6, seed=4,
                                       chain=0, step=k)
        assert st == 0
        assert oracle.membership(A, x_new)
        if refl == 0:
            # no reflection: the end point is Phi(l) of the step's own draws
            v = oracle.gaussians(n, 4, 0, k)
            ell = 3.0 * oracle.uniform(4, 0, k, 1)
            assert np.allclose(x_new, x + v * ell - c / 2.0 * ell ** 2, atol=1e-14)
        x = x_new


def test_fig4_boltzmann_means(example_2d):
    """Fig. 4 (right): the Boltzmann density with T = 1, c = (-0.09, 1) on the
    Appendix B spectrahedron.  The oracle's HMC chains (Alg. 6) reproduce the
    density's mean, computed here by quadrature, within five standard errors
    of their independent end points."""
    A = example_2d
    c, T = np.array([-0.09, 1.0]), 1.0
    mean, var, area = conftest.boltzmann_moments_2d(A, c, T)
    assert abs(area - 10.45) < 0.1  # the area of the reading C1 (Sec. 2.5 example)
    chains, steps = 300, 12
    ends = []
    for ch in range(chains):
        x = np.array([-1.0, 1.0])
        for k in range(steps):
            x, st, _ = hmc.hmc_step(A, x, c, T, tau=6.0, rho=100, kappa=1e-6, seed=21,
                                    chain=ch, step=k)
            assert st == 0
        ends.append(x)
    ends = np.array(ends)
    se = np.sqrt(var / chains)
    assert np.all(np.abs(ends.mean(axis=0) - mean) <= 5 * se), (ends.mean(axis=0), mean, se)
    # the density is not the uniform one: its second moment is pulled down
    assert mean[1] < -0.3


def test_reflection_keeps_the_speed():
    """Reflection on the normal is an isometry: |s| = |Phi'(t+)|, and the
    normal component changes sign (Sec. 2.4)."""
    A = W.ball_random(6, 5, 2.0, seed=W.BASE_SEED + 83)
    g = np.random.default_rng(7)
    for _ in range(5):
        p = g.uniform(-0.2, 0.2, 6)
        v = g.normal(size=6)
        c = g.normal(size=6)
        r = hmc.curve_reflect(A, p, v, c, 0.8)
        assert r["status"] == 0
        vel = v - c / 0.8 * r["t_plus"]
        assert abs(np.linalg.norm(r["s"]) - np.linalg.norm(vel)) <= 1e-12 * np.linalg.norm(vel)
        assert abs(r["s"] @ r["w_hat"] + vel @ r["w_hat"]) <= 1e-12 * np.linalg.norm(vel)


def test_ball_boltzmann_mean_closed_form():
    """exp(-c.x / T) on the unit n-ball: along the unit vector c/|c| the
    marginal is (1 - s^2)^((n-1)/2) exp(-l s), l = |c| / T, whose mean is
    -I_{n/2+1}(l) / I_{n/2}(l) (modified Bessel functions); the oracle's HMC
    chains reproduce it within five standard errors (variance by quadrature)."""
    from scipy import integrate, special
    n, T = 3, 1.0
    c = np.array([1.2, -0.9, 0.0])
    lam = np.linalg.norm(c) / T
    e = c / np.linalg.norm(c)
    mean = -special.iv(n / 2 + 1, lam) / special.iv(n / 2, lam)
    dens = lambda s: (1 - s * s) ** ((n - 1) / 2) * np.exp(-lam * s)
    Z = integrate.quad(dens, -1, 1)[0]
    m2 = integrate.quad(lambda s: s * s * dens(s), -1, 1)[0] / Z
    var = m2 - mean ** 2
    A = W.ball(n, 1.0)
    chains, steps = 400, 10
    ends = []
    for ch in range(chains):
        x = np.zeros(n)
        for k in range(steps):
            x, st, _ = hmc.hmc_step(A, x, c, T, tau=2.0, rho=100, kappa=1e-6, seed=31, chain=ch,
                                    step=k)
            assert st == 0
        ends.append(x @ e)
    ends = np.array(ends)
    se = np.sqrt(var / chains)
    assert abs(ends.mean() - mean) <= 5 * se, (ends.mean(), mean, se)
