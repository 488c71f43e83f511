"""The learned warm start (a network trained on the walk's own refined
oracle outputs) in the Billiard walk.

* Tuples recorded from a mixed-precision walk train the network on the GPU
  (its loss falls).
* The learned walk keeps every invariant (points interior, same moments as
  the oracle's own walk within Monte-Carlo error).
* A/B: with the trained network, stage 1 factors next to the predicted
  boundary point and starts from the predicted null vector, so the stage-1
  Lanczos iteration count per segment drops, while t+ keeps its certified
  refinement.
"""
import math

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


@pytest.fixture(scope="module")
def trained(spectra):
    n = 10
    A = W.ball_random(n, 10, 3.0, seed=W.BASE_SEED + 0)
    m = A.shape[1]
    spec = spectra.Spectrahedron(A)
    tau, tscale = 6.0, 1.0
    net = spectra.MLP(2 * n, 128, 1 + m, seed=1)  # din = 2n = 20
    spec.attach_mlp(net, x_scale=1.0 / 3.0, t_scale=tscale, margin=0.1, iters=12)
    cap = 60000
    X = torch.zeros((cap, 2 * n), dtype=torch.float32, device="cuda")
    Y = torch.zeros((cap, 1 + m), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ch = spectra.Chains(spec, 2048, seed=77)
    ch.record(X, Y, cnt)
    while int(cnt.item()) < cap:
        ch.billiard(2, tau=tau, rho=100, kappa=1e-6, mode="mixed")
    ch.record()
    losses = net.train(X, Y, epochs=30, batch=512, lr=2e-3)
    return dict(spec=spec, A=A, net=net, losses=losses, tau=tau, n=n)


def test_training_reduces_loss(trained):
    losses = trained["losses"]
    assert losses[-1] < 0.5 * losses[0], losses


def test_learned_walk_invariants_and_moments(spectra, trained):
    spec, A, n, tau = trained["spec"], trained["A"], trained["n"], trained["tau"]
    ch = spectra.Chains(spec, 64, seed=31)
    samples = []
    for _ in range(10):
        ch.billiard(100, tau=tau, rho=100, kappa=1e-6, mode="learned")
        x, _ = ch.state()
        assert bool(spec.membership(x).all())
        samples.append(x.cpu().numpy())
    st, stats = ch.status()
    # a step may end at the reflection bound rho (status RHO: a chain caught
    # in a corner of the body, the paper's stopping rule); nothing else fails
    codes = set(np.unique(st.cpu().numpy()).tolist())
    assert codes <= {0, 4}, (stats, codes)
    assert stats["bad_steps"] <= 1e-3 * 64 * 1000, stats
    assert stats["learned_ok"] > 0.5 * stats["segments"], stats
    G = np.concatenate(samples[2:])
    Xo = np.zeros((64, n))
    osamp = []
    for b in range(10):
        Xo, _ = oracle.walk("billiard", A, Xo, 100, tau=tau, rho=100, kappa=1e-6, seed=32,
                            step0=100 * b)
        osamp.append(Xo.copy())
    O = np.concatenate(osamp[2:])
    for fg, fo in [(G, O), ((G ** 2).sum(1, keepdims=True), (O ** 2).sum(1, keepdims=True))]:
        se = np.sqrt(fg.var(0) / len(fg) * 4 + fo.var(0) / len(fo) * 4)
        assert np.all(np.abs(fg.mean(0) - fo.mean(0)) < 5 * se + 1e-12)


def test_learned_first_step_follows_oracle(spectra, trained):
    spec, A, n, tau = trained["spec"], trained["A"], trained["n"], trained["tau"]
    ch = spectra.Chains(spec, 32, seed=11)
    ch.billiard(1, tau=tau, rho=100, kappa=1e-6, mode="learned")
    xs, _ = ch.state()
    Xo, _ = oracle.walk("billiard", A, np.zeros((32, n)), 1, tau=tau, rho=100, kappa=1e-6,
                        seed=11)
    assert np.abs(xs.cpu().numpy() - Xo).max() < 1e-8


def test_warm_start_reduces_stage1_iterations(spectra, trained):
    """A/B test of the network's gain: the same walk with and without it."""
    spec, tau = trained["spec"], trained["tau"]
    res = {}
    for mode in ["mixed", "learned"]:
        ch = spectra.Chains(spec, 1024, seed=5)
        ch.billiard(20, tau=tau, rho=100, kappa=1e-6, mode=mode)
        _, stats = ch.status()
        # stage-1 FP32 Lanczos iterations per segment
        res[mode] = stats["lanczos_iters"] / stats["segments"]
        res[mode + "_stats"] = stats
    assert res["learned"] < 0.8 * res["mixed"], res
