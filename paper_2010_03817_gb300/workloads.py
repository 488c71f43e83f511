"""Seeded synthetic spectrahedra (input generators only).

Each generator returns the LMI stack A of shape (n+1, m, m), float64, with
A[0] = A_0 and A[i] = A_i, so that F(x) = A_0 + sum_i x_i A_i (Eq. 1 of
arXiv 2010.03817).  Nothing here computes any part of the sampling method;
the module serves the GPU library's users, its tests and the oracle's tests
alike.  Seeds follow ``seed = 2010_03817 + workload index``.

Workloads
---------
* :func:`ball_random` -- F(x) = blockdiag([[r, x^T], [x, r I_n]],
  I_k + sum_i x_i S_i), S_i = G_i + G_i^T, G_i entries N(0, 1/(n k)).  The
  first block is the ball |x| <= r (Schur complement); the second is a random
  LMI block.  m = n + 1 + k.
* :func:`rotated_cube` -- F(x) = Q^T diag(1 + x_1, 1 - x_1, ..., 1 + x_n,
  1 - x_n) Q with Q Haar-random orthogonal: the cube [-1, 1]^n, m = 2n.
* :func:`ball` -- the ball block alone, m = n + 1.
* :func:`dabbene` -- the paper's random generator "S-n-m" (Sec. 4):
  A_0 = Z Z^T + I_m with Z ~ U[0, 1]^{m x m}; A_i = blockdiag(Q~, -Q~) with
  Q~ = Q + Q^T, Q ~ U[-1, 1]^{(m/2) x (m/2)}.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 2010_03817


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ball_block(n: int, r: float) -> np.ndarray:
    """Stack (n+1, n+1, n+1) for [[r, x^T], [x, r I_n]] >= 0  <=>  |x| <= r."""
    A = np.zeros((n + 1, n + 1, n + 1))
    A[0] = r * np.eye(n + 1)
    for i in range(1, n + 1):
        A[i, 0, i] = 1.0
        A[i, i, 0] = 1.0
    return A


def random_block(n: int, k: int, seed: int) -> np.ndarray:
    """Stack (n+1, k, k): I_k + sum_i x_i (G_i + G_i^T), G_i ~ N(0, 1/(n k))."""
    g = _rng(seed)
    A = np.zeros((n + 1, k, k))
    A[0] = np.eye(k)
    std = 1.0 / math.sqrt(n * k)
    for i in range(1, n + 1):
        G = g.normal(0.0, std, size=(k, k))
        A[i] = G + G.T
    return A


def blockdiag(*stacks: np.ndarray) -> np.ndarray:
    n1 = stacks[0].shape[0]
    assert all(s.shape[0] == n1 for s in stacks)
    m = sum(s.shape[1] for s in stacks)
    A = np.zeros((n1, m, m))
    o = 0
    for s in stacks:
        k = s.shape[1]
        A[:, o:o + k, o:o + k] = s
        o += k
    return A


def ball_random(n: int, k: int, r: float = 3.0, seed: int = BASE_SEED) -> np.ndarray:
    return blockdiag(ball_block(n, r), random_block(n, k, seed))


def ball(n: int, r: float = 1.0) -> np.ndarray:
    return ball_block(n, r)


def haar_orthogonal(m: int, g: np.random.Generator) -> np.ndarray:
    Z = g.normal(size=(m, m))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def rotated_cube(n: int, seed: int = BASE_SEED) -> np.ndarray:
    m = 2 * n
    Q = haar_orthogonal(m, _rng(seed))
    A = np.zeros((n + 1, m, m))
    A[0] = np.eye(m)
    for i in range(1, n + 1):
        d = np.zeros(m)
        d[2 * (i - 1)] = 1.0
        d[2 * (i - 1) + 1] = -1.0
        A[i] = Q.T @ (d[:, None] * Q)
        A[i] = 0.5 * (A[i] + A[i].T)
    return A


def dabbene(n: int, m: int, seed: int = BASE_SEED) -> np.ndarray:
    if m % 2:
        raise ValueError("the S-n-m generator needs an even m")
    g = _rng(seed)
    h = m // 2
    A = np.zeros((n + 1, m, m))
    Z = g.uniform(0.0, 1.0, size=(m, m))
    A[0] = Z @ Z.T + np.eye(m)
    for i in range(1, n + 1):
        Q = g.uniform(-1.0, 1.0, size=(h, h))
        Qt = Q + Q.T
        A[i, :h, :h] = Qt
        A[i, h:, h:] = -Qt
    return A


def uneven_batch(count: int = 64, lo: int = 20, hi: int = 200, seed: int = BASE_SEED + 3):
    """(n, k) pairs with n, k = round(log-uniform[lo, hi]) for the uneven batch."""
    g = _rng(seed)
    ns = np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(int)
    ks = np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(int)
    return list(zip(ns.tolist(), ks.tolist()))


def random_interior_points(A: np.ndarray, count: int, scale: float, seed: int) -> np.ndarray:
    """`count` points scale * g / |g| * U^(1/n) around the origin (the origin
    is interior for every generator here); callers keep the interior ones."""
    n = A.shape[0] - 1
    g = _rng(seed)
    G = g.normal(size=(count, n))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    rad = scale * g.uniform(0.0, 1.0, size=(count, 1)) ** (1.0 / n)
    return G * rad


def random_directions(n: int, count: int, seed: int) -> np.ndarray:
    g = _rng(seed)
    G = g.normal(size=(count, n))
    return G / np.linalg.norm(G, axis=1, keepdims=True)
