"""Parity of the boundary oracle on the states the Billiard walk actually
visits, at the full size of the benchmark workload: Dabbene S-200-200
(n = m = 200, the generator of Sec. 4), tau = 0.3752, kappa = 1e-6.

Every input here comes from the seeded generators or from the oracle:

- the oracle walks its own chains (Alg. 5) from the start cloud for a few
  steps and traces the lines (p, v) its REFLECTION calls meet -- after a hit
  the next line starts kappa-close to the boundary (reading C4) -- and the
  GPU's sp_reflect is compared with the oracle on exactly those lines, on
  the FP64, mixed and learned paths (t+ to 1e-10 / 1e-9 / 1e-9 relative, the
  unit normal to the same bounds where the eigengap allows, reading C11);
- the GPU walks 8192 chains (the benchmark's launch configuration) from the
  seeded start cloud while recording every boundary-oracle call; the first
  call of every chain has inputs identical to the oracle's (the start point
  and the Philox direction), so its t+ is compared element by element, and
  the first few calls of sampled chains are matched by (chain, step, index)
  with the oracle's own trace of the same chains.
"""
import numpy as np
import pytest

import oracle
from paper_2010_03817_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = M = 200
TAU = 0.3752          # the benchmark's tau for this workload (a pilot chord estimate)
KAPPA, RHO = 1e-6, 1000
SEED_WALK = 1234
TOL_T = {"fp64": 1e-10, "mixed": 1e-9, "learned": 1e-9}
GAP_MIN = 1e-6        # normal parity only where the relative eigengap allows (C11)


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


@pytest.fixture(scope="module")
def workload():
    return W.dabbene(N, M, seed=W.BASE_SEED + 6)


@pytest.fixture(scope="module")
def spec(spectra, workload):
    return spectra.Spectrahedron(workload)


def start_cloud(C):
    return W.random_directions(N, C, seed=SEED_WALK) * 1e-3


@pytest.fixture(scope="module")
def network(spectra, spec):
    """A warm-start network trained on the GPU on tuples the mixed walk
    records (its quality does not matter here: every prediction is checked
    and refined, so the learned path must meet the mixed path's accuracy)."""
    cap = 65536
    X = torch.zeros((cap, 2 * N), dtype=torch.float32, device="cuda")
    Y = torch.zeros((cap, 1 + M), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    spec.attach_mlp(None, x_scale=1.0 / TAU, t_scale=0.05)
    ch = spectra.Chains(spec, 2048, x0=start_cloud(2048), seed=SEED_WALK + 7)
    ch.record(X, Y, cnt)
    ch.billiard(2, tau=TAU, rho=RHO, kappa=KAPPA, mode="mixed")
    ch.record()
    got = min(int(cnt.item()), cap) // 1024 * 1024
    assert got >= 8192
    net = spectra.MLP(2 * N, 512, 1 + M, seed=5)
    net.train(X[:got].contiguous(), Y[:got].contiguous(), epochs=4, batch=1024, lr=1e-3)
    spec.attach_mlp(net, x_scale=1.0 / TAU, t_scale=0.05, margin=0.3, iters=12)
    return net


@pytest.fixture(scope="module")
def visited(workload):
    """Lines the oracle's own Billiard walk meets: 24 chains, two burn-in
    steps from the start cloud, then the traced third step."""
    C = 24
    X, _ = oracle.walk("billiard", workload, start_cloud(C), 2, tau=TAU, rho=RHO, kappa=KAPPA,
                       seed=SEED_WALK)
    _, P, V, st, _ = oracle.billiard_trace(workload, X, 2, tau=TAU, rho=RHO, kappa=KAPPA,
                                           seed=SEED_WALK, max_per_chain=12)
    ref = oracle.reflect_batch(workload, P, V)
    keep = ref["status"] == 0
    return P[keep], V[keep], {k: np.asarray(v)[keep] for k, v in ref.items()}


def _compare(spectra, spec, P, V, ref, mode):
    tp, wh, s, st = spec.reflect(torch.tensor(P, device="cuda"), torch.tensor(V, device="cuda"),
                                 mode=mode)
    tp, wh, s, st = tp.cpu().numpy(), wh.cpu().numpy(), s.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all(), (mode, np.unique(st, return_counts=True))
    et = np.abs(tp - ref["t_plus"]) / np.abs(ref["t_plus"])
    assert et.max() <= TOL_T[mode], (mode, et.max(), int(np.argmax(et)))
    gap = ref["rel_gap"] > GAP_MIN
    ew = np.abs(wh - ref["w_hat"]).max(axis=1)
    assert gap.sum() >= len(P) // 2
    assert ew[gap].max() <= TOL_T[mode], (mode, ew[gap].max())
    # the reflected direction keeps its length and mirrors the normal part
    assert np.allclose(np.linalg.norm(s, axis=1), np.linalg.norm(V, axis=1), rtol=1e-12)
    return et, ew[gap]


def test_visited_lines_are_near_the_boundary(visited):
    """The traced lines include the post-reflection states: starting points
    kappa-close to the boundary, where F(p) is nearly singular."""
    P, V, ref = visited
    assert len(P) >= 64
    # the root behind the point (the boundary just left) is within ~kappa t
    # of it for every line after the first of its step
    close = 0
    for c in range(0, len(P), 7):
        r = oracle.intersect(W.dabbene(N, M, seed=W.BASE_SEED + 6), P[c], V[c])
        close += abs(r["t_minus"]) < 1e-4 * r["t_plus"]
    assert close >= 3


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_reflect_on_visited_lines(spectra, spec, visited, mode):
    P, V, ref = visited
    _compare(spectra, spec, P, V, ref, mode)


def test_learned_reflect_on_visited_lines(spectra, spec, visited, network):
    """The learned path's REFLECTION starts stage 1 from the network's
    prediction on every line (accepted or rejected by its own checks) and
    still meets the 1e-9 bar."""
    P, V, ref = visited
    _compare(spectra, spec, P, V, ref, "learned")
    acc, rej = spec.learned_counts()
    assert acc + rej == len(P), (acc, rej, len(P))


@pytest.mark.parametrize("mode", ["fp64", "mixed", "learned"])
def test_full_size_walk_segments(spectra, spec, workload, network, mode):
    """8192 chains, one Billiard step from the start cloud, every boundary-
    oracle call recorded.  The first call of each chain has exactly the
    oracle's inputs; sampled chains' first calls are matched with the
    oracle's own trace by (chain, step, index)."""
    C = 8192
    n = N
    cap = 8192 * 40
    buf = torch.zeros((cap, 3 * n + 8), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ch = spectra.Chains(spec, C, x0=start_cloud(C), seed=SEED_WALK)
    ch.record_segments(buf, cnt, every=1)
    ch.billiard(1, tau=TAU, rho=RHO, kappa=KAPPA, mode=mode)
    ch.record_segments()
    torch.cuda.synchronize()
    total = int(cnt.item())
    assert total <= cap
    rec = spectra.decode_segments(buf, total, 1, n)
    _, stats = ch.status()
    assert total == stats["segments"]
    assert rec["reflected"].sum() == stats["reflections"]
    # every chain's first call: the start point (the seeded cloud) and its
    # Philox direction, the same inputs as the oracle's (up to the last ulp of
    # the direction: CUDA's and the host's log / sin / cos, reading C13)
    first = np.nonzero(rec["k"] == 0)[0]
    assert len(first) == C
    assert np.array_equal(np.sort(rec["chain"][first]), np.arange(C))
    X0 = start_cloud(C)
    by_chain = {(int(c), int(k)): g for g, (c, k) in enumerate(zip(rec["chain"], rec["k"]))}
    sample = np.arange(0, C, 32)
    Vor = np.stack([oracle.direction(n, SEED_WALK, int(c), 0) for c in sample])
    ref = oracle.reflect_batch(workload, X0[sample], Vor)
    for i, c in enumerate(sample):
        g = by_chain[(int(c), 0)]
        assert np.abs(rec["p"][g] - X0[c]).max() == 0.0
        assert np.abs(rec["v"][g] - Vor[i]).max() < 1e-14
        assert rec["status"][g] == 0
        et = abs(rec["t_plus"][g] - ref["t_plus"][i]) / ref["t_plus"][i]
        assert et <= TOL_T[mode], (mode, int(c), et)
        if rec["reflected"][g] and ref["rel_gap"][i] > GAP_MIN:
            assert np.abs(rec["w_hat"][g] - ref["w_hat"][i]).max() <= TOL_T[mode]
    # later calls of sampled chains, matched by (chain, index) with the
    # oracle's trace of the same chains: after a reflection the two walks'
    # lines differ by rounding only; a shift dp of the line's start moves the
    # hit by (w^.dp)/(w^.v) along it (w^ the normal at the hit point)
    c0, S = 4096, 16
    _, Po, Vo, _, rows = oracle.billiard_trace(workload, X0[c0:c0 + S], 0, tau=TAU, rho=RHO,
                                               kappa=KAPPA, seed=SEED_WALK, chain0=c0,
                                               max_per_chain=4)
    ro = oracle.reflect_batch(workload, Po, Vo)
    matched = 0
    for row in range(len(Po)):
        key = (int(rows["chain"][row]), int(rows["k"][row]))
        if key not in by_chain or ro["status"][row] != 0:
            continue
        g = by_chain[key]
        dp = rec["p"][g] - Po[row]
        assert np.abs(dp).max() < 1e-9, (key, np.abs(dp).max())
        wv = abs(float(ro["w_hat"][row] @ Vo[row]))
        shift = abs(float(ro["w_hat"][row] @ dp)) / max(wv, 1e-3)
        tp = ro["t_plus"][row]
        assert abs(rec["t_plus"][g] - tp) <= TOL_T[mode] * tp + 10.0 * shift, (mode, key)
        matched += 1
    assert matched >= 2 * S
