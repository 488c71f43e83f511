"""Failure detection without a GPU fault: invalid inputs, an exhausted
iteration budget and a garbage warm-start network are injected on the host,
and the library must answer with status words (never a hang or a fault)
while every line it does answer stays within the oracle's tolerance.  Also
bounds the reciprocal routines the dense kernels use in place of the FP64
divide and square root."""
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


def _lines(A, count, seed):
    n = A.shape[0] - 1
    g = np.random.default_rng(seed)
    X = g.uniform(-0.3, 0.3, size=(count, n))
    V = W.random_directions(n, count, seed=seed + 1)
    return X, V


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_nonfinite_lines_get_invalid_status(spectra, mode):
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED)
    spec = spectra.Spectrahedron(A)
    X, V = _lines(A, 8, 3)
    X[1, 4] = np.nan
    V[3, 0] = np.inf
    X[5, 9] = -np.inf
    x, v = torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda")
    tm, tp, _, st = spec.intersect(x, v, mode=mode)
    tp2, wh, s, st2 = spec.reflect(x, v, mode=mode)
    inside = spec.membership(x)
    torch.cuda.synchronize()
    st, st2, tp, tp2 = st.cpu().numpy(), st2.cpu().numpy(), tp.cpu().numpy(), tp2.cpu().numpy()
    bad = [1, 3, 5]
    for c in range(8):
        if c in bad:
            assert st[c] == spectra.ST_INVALID and st2[c] == spectra.ST_INVALID
            assert np.isnan(tp[c]) and np.isnan(tp2[c])
        else:
            assert st[c] == 0 and st2[c] == 0
            r = oracle.reflect(A, X[c], V[c])
            assert abs(tp2[c] - r["t_plus"]) <= 1e-9 * r["t_plus"]
    assert inside.cpu().numpy().tolist() == [1, 0, 1, 1, 1, 0, 1, 1]


def test_iteration_cap_gives_noconv(spectra):
    """kmax = 1: the Lanczos run stops at its cap and the status says so (the
    value is the one-step Ritz estimate, +inf when that step saw no positive
    eigenvalue)."""
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED)
    spec = spectra.Spectrahedron(A)
    X, V = _lines(A, 6, 5)
    x, v = torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda")
    spec.set_solver(kmax=1)
    _, tp, _, st = spec.intersect(x, v)
    assert (st.cpu().numpy() == spectra.ST_NOCONV).all()
    tpn = tp.cpu().numpy()
    assert ((tpn > 0) | np.isinf(tpn)).all()
    spec.set_solver()
    _, tp, _, st = spec.intersect(x, v)
    assert (st.cpu().numpy() == 0).all()
    for c in range(6):
        r = oracle.intersect(A, X[c], V[c])
        assert abs(float(tp[c]) - r["t_plus"]) <= 1e-10 * r["t_plus"]


@pytest.mark.parametrize("garbage", ["overflow", "random"])
def test_garbage_network_cannot_cost_accuracy(spectra, garbage):
    """A warm-start network whose parameters are overwritten with garbage:
    'overflow' makes every prediction non-finite, so every warm start is
    rejected; 'random' makes finite nonsense, which the factorisation, the
    Lanczos test and stage 2 catch.  Either way every result stays within
    1e-9 of the oracle, on the primitive and in the walk."""
    n, k = 12, 20
    A = W.ball_random(n, k, 3.0, seed=W.BASE_SEED + 3)
    m = A.shape[1]
    spec = spectra.Spectrahedron(A)
    net = spectra.MLP(2 * n, 64, 1 + m, seed=1)
    g = np.random.default_rng(9)
    if garbage == "overflow":
        net.set_params(np.full(net.nparams, 3.0e38, dtype=np.float32))
    else:
        net.set_params(g.normal(0.0, 0.05, net.nparams).astype(np.float32))
    spec.attach_mlp(net, x_scale=1.0, t_scale=1.0, margin=0.05, iters=12)
    X, V = _lines(A, 48, 11)
    tp, wh, s, st = spec.reflect(torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda"),
                                 mode="learned")
    acc, rej = spec.learned_counts()
    assert acc + rej == 48
    if garbage == "overflow":
        assert rej == 48
    tp, wh, st = tp.cpu().numpy(), wh.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all()
    for c in range(48):
        r = oracle.reflect(A, X[c], V[c])
        assert abs(tp[c] - r["t_plus"]) <= 1e-9 * r["t_plus"], c
        if r["rel_gap"] > 1e-6:
            assert np.abs(wh[c] - r["w_hat"]).max() <= 1e-9, c
    # the walk with the same network: every step completes inside S
    ch = spectra.Chains(spec, 64, seed=4)
    ch.billiard(3, tau=6.0, rho=100, kappa=1e-6, mode="learned")
    x, _ = ch.state()
    assert bool(spec.membership(x).all())
    _, stats = ch.status()
    assert stats["bad_steps"] == 0
    assert stats["learned_miss"] > 0
    if garbage == "overflow":
        assert stats["learned_ok"] == 0


def test_recip_routines_against_ieee(spectra):
    """The FP32-seeded Newton reciprocals that the Cholesky pivots and the
    diagonal-block inverses use: within 4 ulp of the correctly rounded FP64
    1/sqrt(x) and 1/x over the pivot range [1e-37, 3e37] (the FP64 versions),
    and within 2^-44 relative over [2^-62, 2^100] (the double-float versions:
    below 2^-62 the conversion of x itself keeps only its FP32 part, above
    2^100 the low parts of the intermediate products leave the FP32 normal
    range)."""
    g = np.random.default_rng(0)
    x = np.exp(g.uniform(np.log(1e-37), np.log(3e37), 200000))
    x = np.concatenate([x, [1e-37, 3e37, 1.0, 2.0, 0.5, 1 - 2 ** -53, 1 + 2 ** -52,
                            np.nextafter(1.0, 2.0), 4.0 ** 60, 4.0 ** -60]])
    out = spectra.selftest_recip(torch.tensor(x, device="cuda")).cpu().numpy()
    xl = x.astype(np.longdouble)
    rs = (1 / np.sqrt(xl)).astype(np.float64)
    rc = (1 / xl).astype(np.float64)
    ulp_rs = np.spacing(rs)
    ulp_rc = np.spacing(rc)
    assert (np.abs(out[:, 0] - rs) <= 4 * ulp_rs).all(), np.abs((out[:, 0] - rs) / ulp_rs).max()
    assert (np.abs(out[:, 1] - rc) <= 4 * ulp_rc).all(), np.abs((out[:, 1] - rc) / ulp_rc).max()
    dfr = (x >= 2.0 ** -62) & (x <= 2.0 ** 100)
    assert dfr.sum() > 100000
    assert (np.abs(out[dfr, 2] - rs[dfr]) <= 2.0 ** -44 * rs[dfr]).all()
    assert (np.abs(out[dfr, 3] - rc[dfr]) <= 2.0 ** -44 * rc[dfr]).all()


@pytest.mark.parametrize("ratio", [1.001, 1.2])
def test_warm_start_on_the_second_root(spectra, ratio):
    """Stage 1 is handed the wrong root on purpose: a network whose output is
    the second root's t and exact null vector (all weights zero, the output
    bias set).  On the rotated cube with x = 0 the roots are 1/|v_i| and the
    null vectors are rows of Q, so the right answer is closed-form; the
    factorisation certificates and the dominance of the shift-invert
    iteration (or the FP64 fallback) must still return the first root t+ =
    1/max|v_i| and its face normal."""
    n = 4
    seed = W.BASE_SEED + 60
    A = W.rotated_cube(n, seed=seed)
    m = 2 * n
    Q = W.haar_orthogonal(m, W._rng(seed))
    v = np.array([1.0, 1.0 / ratio, 0.3, -0.2])
    v /= np.linalg.norm(v)
    t_plus, t_2 = 1.0 / v[0], 1.0 / v[1]
    u_2 = Q[3]  # the entry 1 - x_2 - t v_2 of diag(...) vanishes at t_2
    spec = spectra.Spectrahedron(A)
    net = spectra.MLP(2 * n, 16, 1 + m, seed=2)
    flat = np.zeros(net.nparams, dtype=np.float32)
    sizes = [int(np.prod(s)) for _, s in net.layout()]
    b3 = flat[sum(sizes[:5]):]
    b3[0] = np.log(t_2)
    b3[1:1 + m] = u_2
    net.set_params(flat)
    spec.attach_mlp(net, x_scale=1.0, t_scale=1.0, margin=0.05, iters=12)
    X = np.zeros((8, n))
    V = np.tile(v, (8, 1))
    x, vv = torch.tensor(X, device="cuda"), torch.tensor(V, device="cuda")
    pred = net.forward(torch.zeros((8, 2 * n), dtype=torch.float32, device="cuda"))
    assert np.allclose(pred[0, 1:].cpu().numpy(), u_2, atol=1e-7)
    for mode in ["learned", "mixed"]:
        tp, wh, s, st = spec.reflect(x, vv, mode=mode)
        assert (st.cpu().numpy() == 0).all(), mode
        assert np.allclose(tp.cpu().numpy(), t_plus, rtol=1e-9, atol=0.0), (mode, tp, t_plus)
        assert np.allclose(wh.cpu().numpy(), -np.eye(n)[0], atol=1e-9), mode
    acc, rej = spec.learned_counts()
    assert acc + rej == 8
