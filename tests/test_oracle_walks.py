"""Distributional pins for the oracle's walks (Sec. 3: Alg. 4 Hit-and-Run,
CDHR, Alg. 5 Billiard): every walk targets the uniform distribution on S, so
on bodies with known moments the sample moments must agree within their
Monte-Carlo error.  Every emitted point must satisfy F(x) > 0."""
import math

import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W


def _check_cube_uniform(X):
    C, n = X.shape
    se_mean = math.sqrt(1.0 / 3.0 / C)
    assert np.all(np.abs(X.mean(0)) < 4.5 * se_mean)
    # var of U[-1,1] is 1/3; var of the sample variance is (E x^4 - 1/9)/C = (1/5-1/9)/C
    se_var = math.sqrt((1.0 / 5.0 - 1.0 / 9.0) / C)
    assert np.all(np.abs((X ** 2).mean(0) - 1.0 / 3.0) < 4.5 * se_var)
    assert np.all(np.abs(X) < 1.0)


@pytest.mark.parametrize("kind,steps", [("billiard", 25), ("hnr", 40), ("cdhr", 40)])
def test_walk_cube_marginals(kind, steps):
    n, C = 3, 400
    A = W.rotated_cube(n, seed=21)
    X0 = np.zeros((C, n))
    X, stats = oracle.walk(kind, A, X0, steps, tau=2 * math.sqrt(n), rho=100, kappa=1e-6,
                           seed=5)
    assert stats["errors"] == 0
    _check_cube_uniform(X)
    for x in X[:50]:
        assert oracle.membership(A, x)


@pytest.mark.parametrize("kind", ["billiard", "hnr"])
def test_walk_ball_second_moment(kind):
    n, C, R = 4, 400, 1.0
    A = W.ball(n, R)
    X, stats = oracle.walk(kind, A, np.zeros((C, n)), 40, tau=2 * R, rho=100, kappa=1e-6,
                           seed=6)
    assert stats["errors"] == 0
    r2 = (X ** 2).sum(1)
    expect = n * R * R / (n + 2)  # E|x|^2 for the uniform n-ball
    # var of |x|^2 = E r^4 - (E r^2)^2, E r^4 = n R^4/(n+4)
    var = n * R ** 4 / (n + 4) - expect ** 2
    assert abs(r2.mean() - expect) < 4.5 * math.sqrt(var / C)
    assert np.all(r2 < R * R)


def test_billiard_counts_segments_and_reflections():
    n = 3
    A = W.rotated_cube(n, seed=3)
    X, stats = oracle.walk("billiard", A, np.zeros((20, n)), 10, tau=4.0, rho=100, seed=2)
    # a step uses one segment plus one per reflection
    assert stats["segments"] == 20 * 10 + stats["reflections"]
    assert stats["reflections"] > 0


def test_billiard_rho_zero_keeps_point():
    """With rho = 0 any reflection ends the step and the point stays (Alg. 5)."""
    n = 3
    A = W.rotated_cube(n, seed=3)
    x0 = np.array([0.2, -0.1, 0.3])
    stayed = moved = 0
    for step in range(30):
        x, st, nr, ns = oracle.billiard_step(A, x0, 50.0, 0, 1e-6, 9, 0, step)
        if nr > 0:
            assert st == oracle.RHO and np.array_equal(x, x0)
            stayed += 1
        else:
            moved += 1
    assert stayed > 0


def test_billiard_step_is_deterministic_in_counter():
    A = W.ball_random(3, 3, 1.0, seed=1)
    a = oracle.billiard_step(A, np.zeros(3), 1.0, 10, 1e-6, 77, 4, 9)
    b = oracle.billiard_step(A, np.zeros(3), 1.0, 10, 1e-6, 77, 4, 9)
    c = oracle.billiard_step(A, np.zeros(3), 1.0, 10, 1e-6, 77, 5, 9)
    assert np.array_equal(a[0], b[0]) and not np.array_equal(a[0], c[0])


def test_billiard_short_step_is_straight_move():
    """If the drawn length l is below t+ the step is x + l v exactly."""
    n = 3
    A = W.ball(n, 1.0)
    seed, chain, step, tau = 3, 0, 0, 1e-3
    x, st, nr, ns = oracle.billiard_step(A, np.zeros(n), tau, 10, 1e-6, seed, chain, step)
    eta = oracle.uniform(seed, chain, step, 1)
    v = oracle.direction(n, seed, chain, step)
    ell = -tau * math.log(eta)
    assert ell < 1.0 and nr == 0 and ns == 1
    assert np.allclose(x, ell * v, rtol=0, atol=1e-16)


def test_hnr_moves_along_drawn_chord():
    n = 4
    A = W.ball(n, 1.0)
    x0 = np.array([0.1, 0.2, -0.3, 0.0])
    x, st = oracle.hnr_step(A, x0, 4, 2, 6)
    v = oracle.direction(n, 4, 2, 6)
    r = oracle.intersect(A, x0, v)
    eta = oracle.uniform(4, 2, 6, 1)
    t = r["t_minus"] + eta * (r["t_plus"] - r["t_minus"])
    assert np.allclose(x, x0 + t * v, atol=1e-15)


def test_cdhr_moves_one_coordinate():
    n = 4
    A = W.rotated_cube(n, seed=2)
    x0 = np.array([0.1, 0.2, -0.3, 0.0])
    x, st = oracle.cdhr_step(A, x0, 4, 2, 6)
    j = oracle.cdhr_coord(n, 4, 2, 6)
    d = x - x0
    assert np.count_nonzero(d) == 1 and d[j] != 0
    eta = oracle.uniform(4, 2, 6, 1)
    assert x[j] == pytest.approx(-1.0 + eta * 2.0, rel=1e-12)


def test_billiard_trace_follows_alg5():
    """The traced Billiard step is the same step (same end point), and its
    recorded lines chain as Alg. 5 moves: after a hit at t+ the next line
    starts at p + (1 - kappa) t+ v with the reflected direction s."""
    n, kappa = 6, 1e-6
    A = W.ball_random(n, 6, 2.0, seed=W.BASE_SEED + 40)
    X = np.zeros((5, n))
    Xt, P, V, st, rows = oracle.billiard_trace(A, X, 3, tau=4.0, rho=50, kappa=kappa, seed=8,
                                               chain0=2, max_per_chain=64)
    Xw, _ = oracle.walk("billiard", A, X, 1, tau=4.0, rho=50, kappa=kappa, seed=8, step0=3,
                        chain0=2)
    assert np.array_equal(Xt, Xw)
    assert (st == 0).all()
    assert set(rows["chain"]) == set(range(2, 7))
    for i in range(len(P) - 1):
        if rows["chain"][i + 1] != rows["chain"][i]:
            assert rows["k"][i + 1] == 0
            continue
        assert rows["k"][i + 1] == rows["k"][i] + 1
        r = oracle.reflect(A, P[i], V[i])
        assert np.allclose(P[i + 1], P[i] + (1 - kappa) * r["t_plus"] * V[i], atol=1e-14)
        assert np.allclose(V[i + 1], r["s"], atol=1e-14)
    # the first line of each chain: its start point and its Philox direction
    for c in range(5):
        i = int(np.nonzero((rows["chain"] == 2 + c) & (rows["k"] == 0))[0][0])
        assert np.array_equal(P[i], X[c])
        assert np.array_equal(V[i], oracle.direction(n, 8, 2 + c, 3))


def test_reflect_batch_equals_single_calls():
    n = 5
    A = W.rotated_cube(n, seed=W.BASE_SEED + 41)
    g = np.random.default_rng(3)
    P = g.uniform(-0.9, 0.9, size=(7, n))
    V = W.random_directions(n, 7, seed=4)
    rb = oracle.reflect_batch(A, P, V)
    for c in range(7):
        r = oracle.reflect(A, P[c], V[c])
        assert rb["status"][c] == r["status"]
        assert rb["t_plus"][c] == r["t_plus"]
        assert np.array_equal(rb["w_hat"][c], r["w_hat"])
        assert rb["rel_gap"][c] == r["rel_gap"]


def test_intersect_batch_equals_single_calls():
    n = 4
    A = W.ball_random(n, 3, 2.0, seed=W.BASE_SEED + 42)
    g = np.random.default_rng(5)
    P = g.uniform(-0.2, 0.2, size=(6, n))
    V = W.random_directions(n, 6, seed=6)
    rb = oracle.intersect_batch(A, P, V)
    for c in range(6):
        r = oracle.intersect(A, P[c], V[c])
        assert rb["status"][c] == r["status"]
        assert rb["t_plus"][c] == r["t_plus"] and rb["t_minus"][c] == r["t_minus"]
