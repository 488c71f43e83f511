"""Expected value of a function over uniform samples of a spectrahedron
(Sec. 4.2): the Monte Carlo estimator E_N[f] = (1/N) sum_i f(x_i) for the
indicator f = 1(S cap H) of the union of two half-spaces
H = {c.x <= b1} cup {c.x >= b2}, so that E[f] = vol(S cap H) / vol(S).

M independent trials of N chains each start at one point x0 and run a walk
(Hit-and-Run, CDHR or Billiard) for increasing walk lengths; after each
length the estimator of every trial is taken on the GPU
(sp_halfspace_fraction) and the mean and the standard deviation over the M
trials are reported.  The spread over the trials shows how far each walk
has mixed at that length (the paper's variance bound: var(E_N) <= 4 M_eps /
(N eps^2) for a walk with mixing time M_eps).
"""
from __future__ import annotations

import math

import numpy as np

from . import spectra


def study(spec, c, b1: float, b2: float, *, walks=("hnr", "cdhr", "billiard"),
          lengths=(1, 5, 10, 20, 30, 40, 50), trials: int = 20, points: int = 200, x0=None,
          tau: float = 1.0, rho: int = 100, kappa: float = 1e-6, mode: str = "fp64",
          seed: int = 1, truth: float | None = None) -> dict:
    """Run the study; returns {walk: [{"length", "mean", "std", "abs_err"}]}
    (abs_err against `truth` when given)."""
    C = trials * points
    X0 = None if x0 is None else np.tile(np.asarray(x0, dtype=np.float64), (C, 1))
    out = {}
    for w in walks:
        ch = spectra.Chains(spec, C, x0=X0, seed=seed)
        done, rows = 0, []
        for L in lengths:
            k = L - done
            if k > 0:
                if w == "billiard":
                    ch.billiard(k, tau=tau, rho=rho, kappa=kappa, mode=mode)
                elif w == "hnr":
                    ch.hnr(k, mode=mode)
                else:
                    ch.cdhr(k, mode=mode)
            done = L
            fr = ch.halfspace_fraction(c, b1, b2, groups=trials)
            row = {"length": L, "mean": float(fr.mean()), "std": float(fr.std(ddof=1))}
            if truth is not None:
                row["abs_err"] = abs(row["mean"] - truth)
            rows.append(row)
        out[w] = rows
        ch.close()
    return out


def binomial_se(p: float, samples: int) -> float:
    """Standard error of a fraction over `samples` independent points."""
    return math.sqrt(p * (1.0 - p) / samples)
