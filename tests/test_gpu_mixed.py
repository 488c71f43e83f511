"""Mixed-precision path against the FP64 oracle.

* The tensor-core pencil formation (exact digit splitting on BF16 tcgen05):
  V = sum v_j A_j and F(x) = A_0 + sum x_j A_j agree with an FP64 evaluation
  element by element within the truncation of the scheme,
  n 2^-51 max_j |c_j| max_{j>=1} |A_j[p]| (8 digits of 7 bits per operand,
  scaled per coefficient row and per packed entry; A_0 is not split but added
  in FP64), plus the FP64 rounding of the reference and of that addition,
  4 (n+1) 2^-53 sum_j |c_j A_j[p]|.
* INTERSECTION / REFLECTION in mixed mode: t+, t- within 1e-9 relative and
  the unit normal within 1e-9 of the oracle (the mixed path's target after
  its FP64 refinement), on identical (x, v).
* Walks in mixed mode: same invariants and moments as the FP64 path.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_T = 1e-9
TOL_W = 1e-9


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


def _packed(A, c0, c):
    il = np.tril_indices(A.shape[1])
    M = c0 * A[0] + np.tensordot(c, A[1:], axes=1)
    return M[il]


def _abs_packed(A, c0, c):
    il = np.tril_indices(A.shape[1])
    M = abs(c0) * np.abs(A[0]) + np.tensordot(np.abs(c), np.abs(A[1:]), axes=1)
    return M[il]


def _scale_packed(A, c):
    """max_j |c_j| * max_{j>=1} |A_j[p]| (A_0 stays out of the digit split)."""
    il = np.tril_indices(A.shape[1])
    return np.abs(c).max() * np.abs(A[1:]).max(axis=0)[il]


@pytest.mark.parametrize("n,m,count", [(10, 21, 5), (200, 200, 130), (37, 50, 257)])
def test_tensor_core_formation(spectra, n, m, count):
    if m == 21:
        A = W.ball_random(n, m - n - 1, 3.0, seed=1)
    else:
        A = W.dabbene(n, m, seed=2)
    g = np.random.default_rng(3)
    X = g.normal(size=(count, n)) * 0.05
    V = g.normal(size=(count, n))
    V[0] = 0.0  # an all-zero coefficient row
    spec = spectra.Spectrahedron(A)
    x = torch.tensor(X, device="cuda")
    v = torch.tensor(V, device="cuda")
    Fm, Vm = spec.form_pencil(x, v, mode="mixed")
    Fd, Vd = spec.form_pencil(x, v, mode="fp64")
    Fm, Vm, Fd, Vd = (t.cpu().numpy() for t in (Fm, Vm, Fd, Vd))
    for c in list(range(min(count, 6))) + [count - 1]:
        for (got, c0, cc) in [(Fm[c], 1.0, X[c]), (Vm[c], 0.0, V[c])]:
            ref = _packed(A, c0, cc)
            K = A.shape[0]
            bound = ((K - 1) * 2.0 ** -51 * _scale_packed(A, cc)
                     + 4 * K * 2.0 ** -53 * _abs_packed(A, c0, cc) + 1e-300)
            assert np.all(np.abs(got - ref) <= bound), (c, np.max(np.abs(got - ref) / bound))
    # mixed and plain FP64 formation agree everywhere
    assert np.allclose(Fm, Fd, rtol=0, atol=1e-13 * np.abs(Fd).max())
    assert np.allclose(Vm, Vd, rtol=0, atol=1e-13 * np.abs(Vd).max())
    assert np.all(Vm[0] == 0.0)


def _interior_points(A, count, scale, seed):
    for _ in range(30):
        pts = W.random_interior_points(A, 4 * count, scale, seed)
        keep = [p for p in pts if oracle.membership(A, p)]
        if len(keep) >= count:
            return np.array(keep[:count])
        scale *= 0.7
    raise AssertionError("no interior points found")


def _compare_mixed(spectra, A, X, V):
    spec = spectra.Spectrahedron(A)
    x = torch.tensor(X, device="cuda")
    v = torch.tensor(V, device="cuda")
    tm, tp, u, st = spec.intersect(x, v, want_u=True, mode="mixed")
    tp2, wh, s, st2 = spec.reflect(x, v, mode="mixed")
    torch.cuda.synchronize()
    tm, tp, tp2 = tm.cpu().numpy(), tp.cpu().numpy(), tp2.cpu().numpy()
    wh, st, st2 = wh.cpu().numpy(), st.cpu().numpy(), st2.cpu().numpy()
    for c in range(len(X)):
        r = oracle.intersect(A, X[c], V[c])
        rf = oracle.reflect(A, X[c], V[c])
        assert st[c] == 0 and st2[c] == 0, (c, st[c], st2[c])
        assert abs(tp[c] - r["t_plus"]) <= TOL_T * abs(r["t_plus"]), c
        assert abs(tp2[c] - r["t_plus"]) <= TOL_T * abs(r["t_plus"]), c
        assert abs(tm[c] - r["t_minus"]) <= TOL_T * abs(r["t_minus"]), c
        if r["rel_gap"] > 1e-6:
            assert np.abs(wh[c] - rf["w_hat"]).max() <= TOL_W, (c, np.abs(wh[c] - rf["w_hat"]).max())


@pytest.mark.parametrize("n,k", [(10, 10), (12, 52)])
def test_mixed_parity_ball_random(spectra, n, k):
    A = W.ball_random(n, k, 3.0, seed=W.BASE_SEED + n + k)
    X = _interior_points(A, 24, 2.5, seed=1)
    V = W.random_directions(n, 24, seed=2) * 1.7
    _compare_mixed(spectra, A, X, V)


@pytest.mark.parametrize("n,m", [(20, 40), (8, 66)])
def test_mixed_parity_dabbene(spectra, n, m):
    A = W.dabbene(n, m, seed=W.BASE_SEED + 100 + m)
    X = _interior_points(A, 16, 0.02, seed=3)
    V = W.random_directions(n, 16, seed=4)
    _compare_mixed(spectra, A, X, V)


def test_mixed_parity_full_size_sampled(spectra):
    A = W.dabbene(200, 200, seed=W.BASE_SEED + 6)
    X = np.zeros((3, 200))
    X[1:] = W.random_directions(200, 2, seed=9) * 0.03
    V = W.random_directions(200, 3, seed=10)
    _compare_mixed(spectra, A, X, V)


def test_mixed_rotated_cube_closed_form(spectra):
    n = 9
    A = W.rotated_cube(n, seed=W.BASE_SEED + 2)
    g = np.random.default_rng(5)
    X = g.uniform(-0.95, 0.95, size=(32, n))
    V = W.random_directions(n, 32, seed=6)
    spec = spectra.Spectrahedron(A)
    tm, tp, _, st = spec.intersect(torch.tensor(X, device="cuda"),
                                   torch.tensor(V, device="cuda"), mode="mixed")
    tm, tp = tm.cpu().numpy(), tp.cpu().numpy()
    for c in range(32):
        x, v = X[c], V[c]
        up = np.where(v > 0, (1 - x) / v, np.where(v < 0, (-1 - x) / v, np.inf))
        dn = np.where(v < 0, (1 - x) / v, np.where(v > 0, (-1 - x) / v, -np.inf))
        assert tp[c] == pytest.approx(up.min(), rel=TOL_T)
        assert tm[c] == pytest.approx(dn.max(), rel=TOL_T)


def test_mixed_walks_invariants_and_moments(spectra):
    n, C = 5, 2048
    A = W.rotated_cube(n, seed=W.BASE_SEED + 1)
    spec = spectra.Spectrahedron(A)
    for kind in ["billiard", "hnr", "cdhr"]:
        ch = spectra.Chains(spec, C, seed=21)
        if kind == "billiard":
            ch.billiard(20, tau=2 * math.sqrt(n), rho=100, kappa=1e-6, mode="mixed")
        else:
            getattr(ch, kind)(40, mode="mixed")
        x, step = ch.state()
        assert step == (20 if kind == "billiard" else 40)
        assert bool(spec.membership(x).all())
        X = x.cpu().numpy()
        st, stats = ch.status()
        assert stats["bad_steps"] == 0, (kind, stats, np.unique(st.cpu().numpy(),
                                                                return_counts=True))
        se_mean = math.sqrt(1.0 / 3.0 / C)
        se_var = math.sqrt((1.0 / 5.0 - 1.0 / 9.0) / C)
        assert np.all(np.abs(X.mean(0)) < 4.5 * se_mean), kind
        assert np.all(np.abs((X ** 2).mean(0) - 1.0 / 3.0) < 4.5 * se_var), kind


def test_mixed_first_step_follows_oracle(spectra):
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED + 0)
    spec = spectra.Spectrahedron(A)
    for kind in ["billiard", "hnr", "cdhr"]:
        ch = spectra.Chains(spec, 32, seed=11)
        if kind == "billiard":
            ch.billiard(1, tau=6.0, rho=100, kappa=1e-6, mode="mixed")
        else:
            getattr(ch, kind)(1, mode="mixed")
        xs, _ = ch.state()
        Xo, _ = oracle.walk(kind, A, np.zeros((32, n)), 1, tau=6.0, rho=100, kappa=1e-6, seed=11)
        assert np.abs(xs.cpu().numpy() - Xo).max() < 1e-8, kind


def test_mixed_ball_walk_second_moment(spectra):
    n, C, R = 8, 2048, 1.0
    A = W.ball(n, R)
    spec = spectra.Spectrahedron(A)
    ch = spectra.Chains(spec, C, seed=22)
    ch.billiard(25, tau=2 * R, rho=100, kappa=1e-6, mode="mixed")
    x, _ = ch.state()
    assert bool(spec.membership(x).all())
    X = x.cpu().numpy()
    r2 = (X ** 2).sum(1)
    expect = n * R * R / (n + 2)
    var = n * R ** 4 / (n + 4) - expect ** 2
    assert abs(r2.mean() - expect) < 4.5 * math.sqrt(var / C)
