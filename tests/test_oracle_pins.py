"""Pins for the FP64 CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself.

* Philox4x32-10: the known-answer vectors published with the generator
  (Salmon et al., SC 2011, Random123 distribution).
* Cholesky / Jacobi: special cases that reduce to library routines.
* INTERSECTION (Alg. 2): closed forms for the rotated cube and the ball, and
  brute-force bisection on membership (Alg. 1) for tiny random LMIs.
* REFLECTION (Alg. 3, Eq. "reflection"): the closed-form normals of the cube
  faces and the sphere, and the mirror invariants.
* The worked example of Sec. 2.5 / Appendix B and the area in Fig. 4's
  caption (loose: the printed matrices are rounded to one decimal).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize(
    "ctr,key,expect",
    [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ],
)
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key).tolist() == expect


def test_u01_open_interval_and_exact():
    assert oracle.u01(0, 0) == 2.0 ** -53
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # (2k+1) 2^-53 with k = a 2^20 + (b >> 12)
    a, b = 0x12345678, 0x9ABCDEF0
    k = (a << 20) | (b >> 12)
    assert oracle.u01(a, b) == (2 * k + 1) * 2.0 ** -53


def test_gaussian_moments():
    g = np.concatenate([oracle.gaussians(1000, 7, c, 3) for c in range(40)])
    assert abs(g.mean()) < 4.0 / math.sqrt(g.size)
    assert abs(g.var() - 1.0) < 4.0 * math.sqrt(2.0 / g.size)
    # fourth moment of N(0,1) is 3
    assert abs((g ** 4).mean() - 3.0) < 0.15


def test_direction_is_unit_and_isotropic():
    V = np.stack([oracle.direction(5, 11, c, 0) for c in range(4000)])
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    assert np.all(np.abs(V.mean(0)) < 4.0 / math.sqrt(5 * 4000))
    cov = V.T @ V / len(V)
    assert np.allclose(cov, np.eye(5) / 5, atol=0.02)


def test_streams_are_distinct():
    a = oracle.uniform(3, 1, 2, 0)
    b = oracle.uniform(3, 1, 2, 1)
    c = oracle.uniform(3, 1, 3, 1)
    assert len({a, b, c}) == 3


# ---------------------------------------------------------------------------
# linear algebra
# ---------------------------------------------------------------------------
def test_cholesky_matches_library():
    g = np.random.default_rng(1)
    X = g.normal(size=(9, 9))
    F = X @ X.T + 0.1 * np.eye(9)
    L = oracle.cholesky(F)
    assert np.allclose(L, np.linalg.cholesky(F), rtol=1e-13, atol=1e-13)
    assert np.allclose(np.triu(L, 1), 0.0)


def test_cholesky_rejects_indefinite():
    F = np.diag([1.0, 2.0, -1e-12, 3.0])
    assert oracle.cholesky(F) is None
    assert oracle.cholesky(np.diag([1.0, 0.0])) is None


def test_jacobi_matches_library():
    g = np.random.default_rng(2)
    X = g.normal(size=(12, 12))
    S = X + X.T
    ev, Q, sweeps = oracle.jacobi(S)
    assert sweeps > 0
    assert np.allclose(np.sort(ev), np.linalg.eigvalsh(S), rtol=1e-13, atol=1e-13)
    assert np.allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    assert np.allclose(S @ Q, Q * ev[None, :], atol=1e-12)


def test_lmi_is_affine_sum():
    A = W.ball_random(3, 4, 2.0, seed=5)
    x = np.array([0.1, -0.2, 0.3])
    F = oracle.lmi(A, 1.0, x)
    assert np.allclose(F, A[0] + np.tensordot(x, A[1:], axes=1), atol=1e-15)


# ---------------------------------------------------------------------------
# INTERSECTION: closed forms
# ---------------------------------------------------------------------------
def _cube_chord(x, v):
    tp, tm = math.inf, -math.inf
    face = None
    for i in range(len(x)):
        if v[i] > 0:
            a, b = (1 - x[i]) / v[i], (-1 - x[i]) / v[i]
        elif v[i] < 0:
            a, b = (-1 - x[i]) / v[i], (1 - x[i]) / v[i]
        else:
            continue
        if a < tp:
            tp, face = a, i
        tm = max(tm, b)
    return tm, tp, face


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_intersect_rotated_cube(seed):
    n = 7
    A = W.rotated_cube(n, seed=seed)
    g = np.random.default_rng(seed)
    for _ in range(4):
        x = g.uniform(-0.9, 0.9, size=n)
        v = W.random_directions(n, 1, seed * 100 + _)[0]
        r = oracle.intersect(A, x, v)
        tm, tp, face = _cube_chord(x, v)
        assert r["status"] == oracle.OK
        assert r["t_plus"] == pytest.approx(tp, rel=1e-13)
        assert r["t_minus"] == pytest.approx(tm, rel=1e-13)
        rf = oracle.reflect(A, x, v)
        e = np.zeros(n)
        e[face] = -np.sign(v[face])  # inward normal of the face that is hit
        assert np.allclose(rf["w_hat"], e, atol=1e-12)
        s = v.copy()
        s[face] = -s[face]
        assert np.allclose(rf["s"], s, atol=1e-12)


def test_intersect_cube_axis_direction():
    # v with zero entries: only one face pair is reachable
    n = 4
    A = W.rotated_cube(n, seed=9)
    x = np.array([0.5, 0.0, -0.25, 0.0])
    v = np.array([0.0, 0.0, 1.0, 0.0])
    r = oracle.intersect(A, x, v)
    assert r["t_plus"] == pytest.approx(1.25, rel=1e-13)
    assert r["t_minus"] == pytest.approx(-0.75, rel=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_intersect_ball(seed):
    n, R = 6, 1.7
    A = W.ball(n, R)
    g = np.random.default_rng(seed)
    for _ in range(4):
        x = g.uniform(-0.5, 0.5, size=n)
        v = g.normal(size=n) * g.uniform(0.5, 2.0)  # not unit on purpose
        r = oracle.intersect(A, x, v)
        a, b, c = v @ v, x @ v, x @ x - R * R
        disc = math.sqrt(b * b - a * c)
        assert r["t_plus"] == pytest.approx((-b + disc) / a, rel=1e-13)
        assert r["t_minus"] == pytest.approx((-b - disc) / a, rel=1e-13)
        rf = oracle.reflect(A, x, v)
        hit = x + rf["t_plus"] * v
        assert np.allclose(rf["w_hat"], -hit / np.linalg.norm(hit), atol=1e-12)
        assert np.linalg.norm(rf["s"]) == pytest.approx(np.linalg.norm(v), rel=1e-13)


def test_intersect_not_interior():
    A = W.ball(3, 1.0)
    r = oracle.intersect(A, np.array([2.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]))
    assert r["status"] == oracle.NOT_PD


def test_intersect_unbounded_direction():
    # a half-space-like LMI: only x_1 <= 1 constrains the line along e_2
    A = np.zeros((3, 2, 2))
    A[0] = np.eye(2)
    A[1] = np.diag([-1.0, 0.0])
    r = oracle.intersect(A, np.zeros(2), np.array([0.0, 1.0]))
    assert math.isinf(r["t_plus"]) and math.isinf(r["t_minus"])
    rf = oracle.reflect(A, np.zeros(2), np.array([0.0, 1.0]))
    assert rf["status"] == oracle.UNBOUNDED


# ---------------------------------------------------------------------------
# INTERSECTION: brute force on tiny inputs
# ---------------------------------------------------------------------------
def _bisect_boundary(A, x, v, sign):
    lo, hi = 0.0, 1.0
    while oracle.membership(A, x + sign * hi * v):
        lo, hi = hi, 2 * hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        if oracle.membership(A, x + sign * mid * v):
            lo = mid
        else:
            hi = mid
    return sign * lo


@pytest.mark.parametrize("kind", ["ball_random", "dabbene"])
def test_intersect_brute_force(kind):
    for seed in range(3):
        if kind == "ball_random":
            A = W.ball_random(3, 4, 1.5, seed=seed)
        else:
            A = W.dabbene(3, 6, seed=seed)
        n = A.shape[0] - 1
        v = W.random_directions(n, 1, 40 + seed)[0]
        x = np.zeros(n)
        r = oracle.intersect(A, x, v)
        assert r["status"] == oracle.OK
        assert r["t_plus"] == pytest.approx(_bisect_boundary(A, x, v, +1.0), rel=1e-11)
        assert r["t_minus"] == pytest.approx(_bisect_boundary(A, x, v, -1.0), rel=1e-11)


def test_normal_is_gradient_of_det():
    """Lemma "Gradient of det F": w is parallel to grad det F at the hit point
    (central finite differences of det along each axis)."""
    A = W.ball_random(3, 3, 1.2, seed=4)
    x = np.array([0.1, -0.2, 0.05])
    v = W.random_directions(3, 1, 5)[0]
    rf = oracle.reflect(A, x, v)
    p = x + rf["t_plus"] * v
    h = 1e-6
    grad = np.array([
        (np.linalg.det(oracle.lmi(A, 1.0, p + h * e)) - np.linalg.det(oracle.lmi(A, 1.0, p - h * e)))
        / (2 * h) for e in np.eye(3)
    ])
    gh = grad / np.linalg.norm(grad)
    assert abs(abs(gh @ rf["w_hat"]) - 1.0) < 1e-6
    # det grows inward: w (u^T A_j u) points into S
    assert gh @ rf["w_hat"] > 0


# ---------------------------------------------------------------------------
# REFLECTION invariants
# ---------------------------------------------------------------------------
def test_reflection_invariants():
    A = W.ball_random(5, 6, 2.0, seed=8)
    g = np.random.default_rng(8)
    for k in range(5):
        v = g.normal(size=5)
        rf = oracle.reflect(A, np.zeros(5), v)
        wh, s = rf["w_hat"], rf["s"]
        assert np.linalg.norm(wh) == pytest.approx(1.0, rel=1e-14)
        assert np.linalg.norm(s) == pytest.approx(np.linalg.norm(v), rel=1e-13)
        assert s @ wh == pytest.approx(-(v @ wh), rel=1e-12, abs=1e-14)
        # tangential part unchanged
        assert np.allclose(s - (s @ wh) * wh, v - (v @ wh) * wh, atol=1e-13)
        # the ray hits the boundary moving outward: <v, w> < 0 for the inward normal
        assert v @ wh < 0


# ---------------------------------------------------------------------------
# the paper's worked example (Sec. 2.5, Appendix B, Fig. 4) -- loose
# ---------------------------------------------------------------------------
def test_worked_example_2d(example_2d):
    A = example_2d
    p0 = np.array([-1.0, 1.0])
    u = np.array([1.3, 0.8])
    r = oracle.intersect(A, p0, u)
    assert r["status"] == oracle.OK
    assert abs(r["t_plus"] - 0.5) < 0.1
    assert abs(r["t_minus"] + 0.8) < 0.1
    rf = oracle.reflect(A, p0, u)
    w_paper = np.array([-0.2, -1.0]) / math.hypot(0.2, 1.0)
    assert rf["w_hat"] @ w_paper > 0.99
    s_paper = np.array([0.8, -1.3])
    cos = rf["s"] @ s_paper / (np.linalg.norm(rf["s"]) * np.linalg.norm(s_paper))
    assert cos > 0.99
    # the hit point is near the reported (-0.3, 1.4)
    hit = p0 + rf["t_plus"] * u
    assert np.linalg.norm(hit - np.array([-0.3, 1.4])) < 0.15


def test_worked_example_area(example_2d):
    """Fig. 4 reports area 10.23; polar integration of t+ from p0 (loose,
    the matrices are rounded to one decimal)."""
    p0 = np.array([-1.0, 1.0])
    th = np.linspace(0.0, 2 * np.pi, 721)[:-1]
    r = np.array([oracle.intersect(example_2d, p0, np.array([math.cos(t), math.sin(t)]))["t_plus"]
                  for t in th])
    area = 0.5 * np.mean(r ** 2) * 2 * np.pi
    assert abs(area - 10.23) / 10.23 < 0.05
