"""Hamiltonian Monte Carlo with reflections for the Boltzmann density
pi(x) ~ exp(-c.x / T) on a spectrahedron (Sec. 3.3, Alg. 6): the plain,
slow reference of the GPU's degree-2 boundary oracle and walk.

TEST INFRASTRUCTURE ONLY: only the tests may import this module.  It shares
no code with the CUDA path.  numpy's Cholesky, triangular solves and
eigenvalue routines serve as library steps; everything else is written out.

For f(x) = c.x / T the Hamiltonian ODE (Eq. ode_ham: dp/dt = v, dv/dt =
-grad f) has the exact degree-2 solution Phi(t) = p + v t - (c / (2T)) t^2,
so F(Phi(t)) = F(p) + t V + t^2 C with V = sum v_j A_j and
C = -(1/(2T)) sum c_j A_j: a quadratic eigenvalue problem (Sec. 2.1).  Its
first positive root comes from the companion linearisation (Sec. 2.1): with
F(p) = L L^T, B = L^{-1} V L^{-T} and K = L^{-1} C L^{-T}, the roots t = 1/mu
for the eigenvalues mu of [[0, I], [-K, -B]] (size 2m); the first root is
1/mu for the largest real positive mu.  It is refined (within 1e-7 relative) by the scalar quadratic
u^T F(Phi(t)) u = 0 with u the null vector of F(Phi(t+)) (stationary at u).
The reflection (Sec. 2.4 for a curve): s = Phi'(t+) - 2 <Phi'(t+), w^> w^,
w_j = u^T A_j u the normal at the hit point.
"""
from __future__ import annotations

import numpy as np

from . import gaussians, lmi, uniform

OK, NOT_PD, UNBOUNDED, RHO, DEGENERATE = 0, 1, 2, 4, 5


def curve_matrices(A, p, v, c, T):
    """F(p), V and C of the trajectory Phi(t) = p + v t - (c/(2T)) t^2."""
    F = lmi(A, 1.0, p)
    V = lmi(A, 0.0, v)
    C = -lmi(A, 0.0, np.asarray(c, dtype=np.float64)) / (2.0 * T)
    return F, V, C


def curve_roots(A, p, v, c, T, imag_tol=1e-10):
    """The real positive roots of det F(Phi(t)), ascending, from the
    companion eigenvalues (None if F(p) is not positive definite)."""
    F, V, C = curve_matrices(A, p, v, c, T)
    m = F.shape[0]
    try:
        L = np.linalg.cholesky(F)
    except np.linalg.LinAlgError:
        return None
    Li = np.linalg.inv(L)
    B = Li @ V @ Li.T
    K = Li @ C @ Li.T
    G = np.zeros((2 * m, 2 * m))
    G[:m, m:] = np.eye(m)
    G[m:, :m] = -K
    G[m:, m:] = -B
    mu = np.linalg.eigvals(G)
    real = mu[(np.abs(mu.imag) <= imag_tol * np.abs(mu)) & (mu.real > 0)].real
    return np.sort(1.0 / real)


def _null_vector(M):
    """Unit eigenvector of the symmetric M for its eigenvalue of least
    magnitude, largest-magnitude entry positive."""
    w, Q = np.linalg.eigh(M)
    u = Q[:, int(np.argmin(np.abs(w)))]
    big = int(np.argmax(np.abs(u)))
    return u * (1.0 if u[big] >= 0 else -1.0)


def curve_reflect(A, p, v, c, T):
    """REFLECTION of the degree-2 trajectory: t+, the unit normal w^ at
    Phi(t+), the reflected velocity s and the status."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0] - 1
    p, v, c = (np.asarray(a, dtype=np.float64) for a in (p, v, c))
    roots = curve_roots(A, p, v, c, T)
    if roots is None:
        return dict(status=NOT_PD, t_plus=0.0, w_hat=np.zeros(n), s=np.zeros(n))
    if len(roots) == 0:
        return dict(status=UNBOUNDED, t_plus=np.inf, w_hat=np.zeros(n), s=np.zeros(n))
    t = roots[0]
    F, V, C = curve_matrices(A, p, v, c, T)
    u = _null_vector(F + t * V + t * t * C)
    # refine t on the scalar quadratic a + b t + c t^2 = 0 (the root nearest t)
    a, b, cc = u @ F @ u, u @ V @ u, u @ C @ u
    if abs(cc) > 0:
        r = np.roots([cc, b, a])
        r = r[np.abs(r.imag) == 0].real if np.iscomplexobj(r) else r
    else:
        r = np.array([-a / b])
    if len(r):
        tr = r[np.argmin(np.abs(r - t))]
        if abs(tr - t) <= 1e-7 * t:
            t = tr
            u = _null_vector(F + t * V + t * t * C)
    w = np.array([u @ A[j] @ u for j in range(1, n + 1)])
    nw = np.linalg.norm(w)
    if not nw > 0:
        return dict(status=DEGENERATE, t_plus=t, w_hat=np.zeros(n), s=np.zeros(n))
    wh = w / nw
    vel = v - (c / T) * t
    s = vel - 2.0 * (vel @ wh) * wh
    return dict(status=OK, t_plus=t, w_hat=wh, s=s)


def hmc_step(A, x, c, T, *, tau, rho, kappa, seed, chain, step):
    """One step of Alg. 6: l = tau eta, v ~ N(0, I_n) (the oracle's Philox
    stream 0 Gaussians, not normalised), then reflections until l is used
    up; after a hit at t+ the walker sits at Phi((1 - kappa) t+) with the
    reflected velocity.  More than rho reflections keep x (status RHO).
    Returns (x_new, status, reflections)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0] - 1
    c = np.asarray(c, dtype=np.float64)
    v = gaussians(n, seed, chain, step)
    ell = tau * uniform(seed, chain, step, 1)
    p = np.array(x, dtype=np.float64)
    refl = 0
    while True:
        r = curve_reflect(A, p, v, c, T)
        if r["status"] != OK:
            return np.array(x, dtype=np.float64), r["status"], refl
        t = r["t_plus"]
        if t < ell:
            tb = (1.0 - kappa) * t
            p = p + v * tb - (c / (2.0 * T)) * tb * tb
            v = r["s"]
            ell -= t
            refl += 1
            if refl > rho:
                return np.array(x, dtype=np.float64), RHO, refl
        else:
            return p + v * ell - (c / (2.0 * T)) * ell * ell, OK, refl
