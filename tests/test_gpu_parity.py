"""GPU <-> oracle parity of the boundary oracle (Alg. 2 INTERSECTION, Alg. 3
REFLECTION, Alg. 1 MEMBERSHIP) on identical (x, v), through the C ABI.

Tolerance of the FP64 path: 1e-10 relative on t+ / t- and 1e-10 on the unit
normal and the reflected direction (absolute, they are unit-scale), cases
whose relative eigengap is below 1e-6 excepted for the normal (the null
vector is then not unique; the oracle reports the gap).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_T = 1e-10
TOL_W = 1e-10


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


def _interior_points(A, count, scale, seed):
    """`count` interior points: a random cloud shrunk until enough are inside."""
    for _ in range(30):
        pts = W.random_interior_points(A, 4 * count, scale, seed)
        keep = [p for p in pts if oracle.membership(A, p)]
        if len(keep) >= count:
            return np.array(keep[:count])
        scale *= 0.7
    raise AssertionError("no interior points found")


def _compare(spectra, A, X, V, check_w=True):
    spec = spectra.Spectrahedron(A)
    x = torch.tensor(X, device="cuda")
    v = torch.tensor(V, device="cuda")
    tm, tp, u, st = spec.intersect(x, v, want_u=True)
    tp2, wh, s, st2 = spec.reflect(x, v)
    torch.cuda.synchronize()
    tm, tp, tp2 = tm.cpu().numpy(), tp.cpu().numpy(), tp2.cpu().numpy()
    wh, s, st, st2 = wh.cpu().numpy(), s.cpu().numpy(), st.cpu().numpy(), st2.cpu().numpy()
    worst = dict(t_plus=0.0, t_minus=0.0, w=0.0)
    for c in range(len(X)):
        r = oracle.intersect(A, X[c], V[c])
        rf = oracle.reflect(A, X[c], V[c])
        assert r["status"] == 0 and st[c] == 0 and st2[c] == 0, (c, r["status"], st[c], st2[c])
        et = abs(tp[c] - r["t_plus"]) / abs(r["t_plus"])
        em = abs(tm[c] - r["t_minus"]) / abs(r["t_minus"])
        et2 = abs(tp2[c] - rf["t_plus"]) / abs(rf["t_plus"])
        worst["t_plus"] = max(worst["t_plus"], et, et2)
        worst["t_minus"] = max(worst["t_minus"], em)
        assert et <= TOL_T and et2 <= TOL_T, (c, et, et2)
        assert em <= TOL_T, (c, em)
        if check_w and r["rel_gap"] > 1e-6:
            ew = np.abs(wh[c] - rf["w_hat"]).max()
            es = np.abs(s[c] - rf["s"]).max() / np.linalg.norm(V[c])
            worst["w"] = max(worst["w"], ew, es)
            assert ew <= TOL_W and es <= TOL_W, (c, ew, es)
    spec.close()
    return worst


@pytest.mark.parametrize("n,k", [(10, 10), (6, 27), (12, 52)])
def test_parity_ball_random(spectra, n, k):
    A = W.ball_random(n, k, 3.0, seed=W.BASE_SEED + n + k)
    X = _interior_points(A, 24, 2.5, seed=1)
    V = W.random_directions(n, 24, seed=2) * 1.7
    _compare(spectra, A, X, V)


@pytest.mark.parametrize("n,m", [(4, 6), (20, 40), (8, 66)])
def test_parity_dabbene(spectra, n, m):
    A = W.dabbene(n, m, seed=W.BASE_SEED + 100 + m)
    X = _interior_points(A, 16, 0.02, seed=3)
    V = W.random_directions(n, 16, seed=4)
    _compare(spectra, A, X, V)


def test_rotated_cube_closed_form(spectra):
    n = 9
    A = W.rotated_cube(n, seed=W.BASE_SEED + 2)
    g = np.random.default_rng(5)
    X = g.uniform(-0.95, 0.95, size=(32, n))
    V = W.random_directions(n, 32, seed=6)
    spec = spectra.Spectrahedron(A)
    tm, tp, _, st = spec.intersect(torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda"))
    tp2, wh, s, st2 = spec.reflect(torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda"))
    tm, tp, wh = tm.cpu().numpy(), tp.cpu().numpy(), wh.cpu().numpy()
    for c in range(32):
        x, v = X[c], V[c]
        up = np.where(v > 0, (1 - x) / v, np.where(v < 0, (-1 - x) / v, np.inf))
        dn = np.where(v < 0, (1 - x) / v, np.where(v > 0, (-1 - x) / v, -np.inf))
        face = int(np.argmin(up))
        assert tp[c] == pytest.approx(up.min(), rel=TOL_T)
        assert tm[c] == pytest.approx(dn.max(), rel=TOL_T)
        e = np.zeros(n)
        e[face] = -np.sign(v[face])
        assert np.abs(wh[c] - e).max() <= TOL_W


def test_ball_closed_form(spectra):
    n, R = 16, 1.3
    A = W.ball(n, R)
    g = np.random.default_rng(7)
    X = g.uniform(-0.3, 0.3, size=(16, n))
    V = g.normal(size=(16, n))
    spec = spectra.Spectrahedron(A)
    tm, tp, _, st = spec.intersect(torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda"))
    tm, tp = tm.cpu().numpy(), tp.cpu().numpy()
    for c in range(16):
        x, v = X[c], V[c]
        a, b, cc = v @ v, x @ v, x @ x - R * R
        d = math.sqrt(b * b - a * cc)
        assert tp[c] == pytest.approx((-b + d) / a, rel=TOL_T)
        assert tm[c] == pytest.approx((-b - d) / a, rel=TOL_T)


def test_parity_full_size_sampled(spectra):
    """Dabbene S-200-200 (n = m = 200) at full size: sampled items against the oracle."""
    A = W.dabbene(200, 200, seed=W.BASE_SEED + 6)
    g = np.random.default_rng(8)
    X = np.zeros((3, 200))
    X[1:] = W.random_directions(200, 2, seed=9) * 0.03
    assert all(oracle.membership(A, x) for x in X)
    V = W.random_directions(200, 3, seed=10)
    _compare(spectra, A, X, V)


def test_membership(spectra):
    A = W.ball(3, 1.0)
    X = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [0.6, 0.6, 0.6], [2.0, 0.0, 0.0]])
    spec = spectra.Spectrahedron(A)
    inside = spec.membership(torch.tensor(X, device="cuda")).cpu().numpy()
    assert inside.tolist() == [int(oracle.membership(A, x)) for x in X] == [1, 1, 0, 0]


def test_edge_cases(spectra):
    A = W.ball(3, 1.0)
    spec = spectra.Spectrahedron(A)
    # empty batch
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    tm, tp, _, st = spec.intersect(e, e)
    assert tm.numel() == 0
    # point outside S
    f64 = dict(dtype=torch.float64, device="cuda")
    x = torch.tensor([[2.0, 0.0, 0.0]], **f64)
    v = torch.tensor([[1.0, 0.0, 0.0]], **f64)
    _, _, _, st = spec.intersect(x, v)
    assert int(st[0]) == spectra.ST_NOT_PD
    # a half-space-like LMI: the ray along e_2 never hits the boundary
    H = np.zeros((3, 2, 2))
    H[0] = np.eye(2)
    H[1] = np.diag([-1.0, 0.0])
    sh = spectra.Spectrahedron(H)
    _, tp, _, st = sh.reflect(torch.zeros((1, 2), dtype=torch.float64, device="cuda"),
                              torch.tensor([[0.0, 1.0]], **f64))
    assert int(st[0]) == spectra.ST_UNBOUNDED
    # m = 1 (a single linear inequality) and n = 1
    L1 = np.array([[[2.0]], [[-1.0]], [[0.5]]])  # 2 - x1 + 0.5 x2 >= 0
    s1 = spectra.Spectrahedron(L1)
    _, tp, _, st = s1.intersect(torch.zeros((1, 2), dtype=torch.float64, device="cuda"),
                                torch.tensor([[1.0, 0.0]], **f64))
    assert int(st[0]) == 0 and float(tp[0]) == pytest.approx(2.0, rel=1e-14)
    B1 = W.ball(1, 2.0)
    sb = spectra.Spectrahedron(B1)
    tm, tp, _, st = sb.intersect(torch.tensor([[0.5]], **f64),
                                 torch.tensor([[1.0]], **f64))
    assert float(tp[0]) == pytest.approx(1.5, rel=1e-14)
    assert float(tm[0]) == pytest.approx(-2.5, rel=1e-14)


def test_bad_arguments(spectra):
    with pytest.raises(spectra.SpectraError):
        spectra.Spectrahedron(np.array([[[1.0, 2.0], [0.0, 1.0]]] * 2))  # not symmetric
    spec = spectra.Spectrahedron(W.ball(2, 1.0))
    with pytest.raises(spectra.SpectraError):
        spectra.Chains(spec, 2, x0=np.array([[0.0, 0.0], [3.0, 0.0]]), seed=1)  # not interior
