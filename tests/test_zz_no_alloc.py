"""The allocation-free INTERSECTION entry point (for callers that cannot
allocate device memory) gives the results of the regular entry point.

It is called twice in a row on the same inputs, through the C ABI, and both
calls must agree with sp_intersect within the FP64 parity tolerance of the
other GPU tests (1e-10 relative on t+ and t-), while the device's free
memory stays exactly where it was (the entry point allocates nothing).
This file sorts last so that a stop-at-first-failure run has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_T = 1e-10


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


@pytest.mark.parametrize("kind", ["ball_random", "dabbene"])
def test_noalloc_matches_intersect(spectra, kind):
    if kind == "ball_random":
        A = W.ball_random(10, 10, 3.0, seed=W.BASE_SEED)
        X = W.random_directions(10, 40, seed=1) * 0.5
    else:
        A = W.dabbene(30, 60, seed=W.BASE_SEED + 50)
        X = W.random_directions(30, 40, seed=1) * 0.002
    n, m = A.shape[0] - 1, A.shape[1]
    V = W.random_directions(n, 40, seed=2)
    x = torch.tensor(X, device="cuda")
    v = torch.tensor(V, device="cuda")
    spec = spectra.Spectrahedron(A)
    tm_ref, tp_ref, _, st_ref = spec.intersect(x, v)
    Ap = torch.tensor(spectra.pack_lmi(A), device="cuda")
    outs = [(torch.empty(40, dtype=torch.float64, device="cuda"),
             torch.empty(40, dtype=torch.float64, device="cuda"),
             torch.empty(40, dtype=torch.int32, device="cuda")) for _ in range(3)]
    for tm, tp, st in outs:
        tm.fill_(float("nan"))
        tp.fill_(float("nan"))
        st.fill_(-1)
    # a first call (it looks up the array's address on this device and loads
    # the kernels), then the device's free memory must not move across the two
    # checked calls: every buffer is allocated and filled already, and nothing
    # else runs in between
    spectra.intersect_noalloc(Ap, n, m, x, v, *outs[2])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        spectra.intersect_noalloc(Ap, n, m, x, v, *outs[call])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for call in range(2):
        tm, tp, st = outs[call]
        assert torch.equal(st, st_ref), call
        assert bool((st == 0).all())
        assert torch.allclose(tp, tp_ref, rtol=TOL_T, atol=0.0), call
        assert torch.allclose(tm, tm_ref, rtol=TOL_T, atol=0.0), call


def test_noalloc_rejects_oversized(spectra):
    n, m = 4, 400  # the factor of m = 400 does not fit one block's shared memory
    Ap = torch.zeros((n + 1, m * (m + 1) // 2), dtype=torch.float64, device="cuda")
    x = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(spectra.SpectraError) as e:
        spectra.intersect_noalloc(Ap, n, m, x, x, out, out.clone(), st)
    assert e.value.code == spectra.EINVAL
