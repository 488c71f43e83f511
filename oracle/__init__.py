"""FP64 CPU oracle (test infrastructure).

This package is the slow, plain reference implementation that the GPU library
is checked against: full m x m matrices, textbook Cholesky, a cyclic Jacobi
eigensolver, Philox4x32-10, and the walks of Sec. 3 (Alg. 4 Hit-and-Run,
CDHR, Alg. 5 Billiard) of arXiv 2010.03817.  It shares no code with the CUDA
path.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import it; the product never does.

The C source is ``oracle/spectra_oracle.c``; :func:`build` compiles it with
gcc into ``oracle/_build/liboracle.so`` (OpenMP over chains when available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spectra_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

# status codes of the oracle (its own, independent of the GPU library's)
OK, NOT_PD, UNBOUNDED, NOCONV, RHO, DEGENERATE, EINVAL = range(7)

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, so both
    host architectures round the same way).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o",
            _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_u01.restype = ctypes.c_double
            L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_gaussians.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, _dp]
            L.orc_direction.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, _dp]
            L.orc_lmi.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp, _dp]
            L.orc_cholesky.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_cholesky.restype = ctypes.c_int
            L.orc_membership.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.orc_membership.restype = ctypes.c_int
            L.orc_jacobi.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int]
            L.orc_jacobi.restype = ctypes.c_int
            L.orc_intersect.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                        _dp, _dp, _dp, _dp]
            L.orc_intersect.restype = ctypes.c_int
            L.orc_reflect.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                      _dp, _dp]
            L.orc_reflect.restype = ctypes.c_int
            L.orc_billiard_step.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            _i32p, _i32p]
            L.orc_billiard_step.restype = ctypes.c_int
            L.orc_hnr_step.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32]
            L.orc_hnr_step.restype = ctypes.c_int
            L.orc_cdhr_step.argtypes = L.orc_hnr_step.argtypes
            L.orc_cdhr_step.restype = ctypes.c_int
            L.orc_cdhr_coord.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_uint32]
            L.orc_cdhr_coord.restype = ctypes.c_int
            L.orc_walk.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                   _dp, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_uint64, _i64p]
            L.orc_walk.restype = ctypes.c_int
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_billiard_trace.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                             ctypes.c_int, _dp, _dp, _i32p, _i32p]
            L.orc_billiard_trace.restype = None
            L.orc_reflect_batch.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                            _dp, _dp, _dp, _dp, _i32p, _dp]
            L.orc_reflect_batch.restype = None
            L.orc_intersect_batch.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                              _dp, _dp, _dp, _i32p]
            L.orc_intersect_batch.restype = None
            _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _stack(A) -> tuple[np.ndarray, int, int]:
    A = _f64(A)
    if A.ndim != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("A must be (n+1) x m x m")
    return A, A.shape[0] - 1, A.shape[1]


# ----------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p),
                            out.ctypes.data_as(_u32p))
    return out


def u01(a: int, b: int) -> float:
    return lib().orc_u01(a, b)


def uniform(seed: int, chain: int, step: int, stream: int) -> float:
    return lib().orc_uniform(seed, chain, step, stream)


def gaussians(n: int, seed: int, chain: int, step: int) -> np.ndarray:
    g = np.zeros(n)
    lib().orc_gaussians(n, seed, chain, step, _d(g))
    return g


def direction(n: int, seed: int, chain: int, step: int) -> np.ndarray:
    v = np.zeros(n)
    lib().orc_direction(n, seed, chain, step, _d(v))
    return v


def cdhr_coord(n: int, seed: int, chain: int, step: int) -> int:
    return lib().orc_cdhr_coord(n, seed, chain, step)


# ----------------------------------------------------------------------------
# linear algebra and the geometric operations
# ----------------------------------------------------------------------------
def lmi(A, c0: float, c) -> np.ndarray:
    A, n, m = _stack(A)
    c = _f64(c)
    out = np.zeros((m, m))
    lib().orc_lmi(n, m, _d(A), c0, _d(c), _d(out))
    return out


def cholesky(F):
    """Lower Cholesky factor, or None if F is not positive definite."""
    F = _f64(F)
    m = F.shape[0]
    L = np.zeros((m, m))
    r = lib().orc_cholesky(m, _d(F), _d(L))
    return None if r else L


def jacobi(S, max_sweeps: int = 100):
    """Eigenvalues and eigenvectors (columns) of a symmetric matrix."""
    S = _f64(S).copy()
    m = S.shape[0]
    ev = np.zeros(m)
    Q = np.zeros((m, m))
    sweeps = lib().orc_jacobi(m, _d(S), _d(ev), _d(Q), max_sweeps)
    return ev, Q, sweeps


def membership(A, x) -> bool:
    A, n, m = _stack(A)
    return bool(lib().orc_membership(n, m, _d(A), _d(_f64(x))))


def intersect(A, x, v) -> dict:
    """Alg. 2 for the line x + t v: t-, t+, unit null vectors, quadratic forms
    w_j = u+^T A_j u+ (j = 0..n) and the oracle's error bar."""
    A, n, m = _stack(A)
    x, v = _f64(x), _f64(v)
    tm = np.zeros(1)
    tp = np.zeros(1)
    up = np.zeros(m)
    um = np.zeros(m)
    wp = np.zeros(n + 1)
    info = np.zeros(4)
    st = lib().orc_intersect(n, m, _d(A), _d(x), _d(v), _d(tm), _d(tp), _d(up), _d(um),
                             _d(wp), _d(info))
    return dict(status=st, t_minus=tm[0], t_plus=tp[0], u_plus=up, u_minus=um, w_forms=wp,
                err_bar=info[0], rel_gap=info[1], sweeps=int(info[2]), err_bar_minus=info[3])


def reflect(A, x, v) -> dict:
    """Alg. 3: t+, unit normal w^ (w_j = u^T A_j u, j = 1..n) and the reflected
    direction s = v - 2 <v, w^> w^."""
    A, n, m = _stack(A)
    x, v = _f64(x), _f64(v)
    tp = np.zeros(1)
    wh = np.zeros(n)
    s = np.zeros(n)
    info = np.zeros(4)
    st = lib().orc_reflect(n, m, _d(A), _d(x), _d(v), _d(tp), _d(wh), _d(s), _d(info))
    return dict(status=st, t_plus=tp[0], w_hat=wh, s=s, err_bar=info[0], rel_gap=info[1])


# ----------------------------------------------------------------------------
# walks
# ----------------------------------------------------------------------------
def billiard_step(A, x, tau: float, rho: int, kappa: float, seed: int, chain: int, step: int):
    A, n, m = _stack(A)
    x = _f64(x).copy()
    nr = ctypes.c_int(0)
    ns = ctypes.c_int(0)
    st = lib().orc_billiard_step(n, m, _d(A), _d(x), tau, rho, kappa, seed, chain, step,
                                 ctypes.byref(nr), ctypes.byref(ns))
    return x, st, nr.value, ns.value


def hnr_step(A, x, seed: int, chain: int, step: int):
    A, n, m = _stack(A)
    x = _f64(x).copy()
    st = lib().orc_hnr_step(n, m, _d(A), _d(x), seed, chain, step)
    return x, st


def cdhr_step(A, x, seed: int, chain: int, step: int):
    A, n, m = _stack(A)
    x = _f64(x).copy()
    st = lib().orc_cdhr_step(n, m, _d(A), _d(x), seed, chain, step)
    return x, st


WALKS = {"billiard": 0, "hnr": 1, "cdhr": 2}


def walk(kind: str, A, X, steps: int, *, tau: float = 1.0, rho: int = 100, kappa: float = 1e-6,
         seed: int = 0, step0: int = 0, chain0: int = 0):
    """Run `steps` steps on every row of X (C x n, copied).  Returns
    (X_new, dict(segments, reflections, bad_steps, errors))."""
    A, n, m = _stack(A)
    X = _f64(X).copy()
    C = X.shape[0]
    counts = np.zeros(3, dtype=np.int64)
    err = lib().orc_walk(WALKS[kind], n, m, _d(A), C, _d(X), steps, step0, chain0, tau, rho,
                         kappa, seed, counts.ctypes.data_as(_i64p))
    return X, dict(segments=int(counts[0]), reflections=int(counts[1]),
                   bad_steps=int(counts[2]), errors=int(err))


def billiard_trace(A, X, step: int, *, tau: float, rho: int = 100, kappa: float = 1e-6,
                   seed: int = 0, chain0: int = 0, max_per_chain: int = 64):
    """One Billiard step (Alg. 5) of every row of X (C x n, copied), recording
    the line (p, v) of each segment the boundary oracle is called on.
    Returns (X_new, P, V, status, rows): P and V are (K x n) stacks of the
    recorded lines, in chain order (at most max_per_chain per chain), status
    the per-chain step statuses, and rows a dict of per-row labels "chain"
    (the Philox chain index chain0 + c) and "k" (index within the step)."""
    A, n, m = _stack(A)
    X = _f64(X).copy()
    C = X.shape[0]
    rp = np.zeros((C * max_per_chain, n))
    rv = np.zeros((C * max_per_chain, n))
    nseg = np.zeros(C, dtype=np.int32)
    status = np.zeros(C, dtype=np.int32)
    lib().orc_billiard_trace(n, m, _d(A), C, _d(X), step, chain0, tau, rho, kappa, seed,
                             max_per_chain, _d(rp), _d(rv), nseg.ctypes.data_as(_i32p),
                             status.ctypes.data_as(_i32p))
    counts = [min(int(nseg[c]), max_per_chain) for c in range(C)]
    keep = np.concatenate([np.arange(c * max_per_chain, c * max_per_chain + counts[c])
                           for c in range(C)])
    rows = {"chain": np.concatenate([np.full(counts[c], chain0 + c) for c in range(C)]),
            "k": np.concatenate([np.arange(counts[c]) for c in range(C)])}
    return X, rp[keep], rv[keep], status, rows


def reflect_batch(A, P, V) -> dict:
    """reflect() on every line (P[c], V[c]) (count x n each), in parallel."""
    A, n, m = _stack(A)
    P, V = _f64(P), _f64(V)
    cnt = P.shape[0]
    tp = np.zeros(cnt)
    wh = np.zeros((cnt, n))
    s = np.zeros((cnt, n))
    st = np.zeros(cnt, dtype=np.int32)
    info = np.zeros((cnt, 4))
    lib().orc_reflect_batch(n, m, _d(A), cnt, _d(P), _d(V), _d(tp), _d(wh), _d(s),
                            st.ctypes.data_as(_i32p), _d(info))
    return dict(status=st, t_plus=tp, w_hat=wh, s=s, err_bar=info[:, 0], rel_gap=info[:, 1])


def intersect_batch(A, P, V) -> dict:
    """intersect() (t-, t+, status) on every line (P[c], V[c]), in parallel."""
    A, n, m = _stack(A)
    P, V = _f64(P), _f64(V)
    cnt = P.shape[0]
    tm = np.zeros(cnt)
    tp = np.zeros(cnt)
    st = np.zeros(cnt, dtype=np.int32)
    lib().orc_intersect_batch(n, m, _d(A), cnt, _d(P), _d(V), _d(tm), _d(tp),
                              st.ctypes.data_as(_i32p))
    return dict(status=st, t_minus=tm, t_plus=tp)


def num_threads() -> int:
    return lib().orc_num_threads()
