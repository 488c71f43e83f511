"""Pin of the CPU reference of the warm-start network (oracle/mlp.py): its
analytic gradients against central finite differences on a tiny network."""
import numpy as np

from oracle import mlp


def test_reference_gradients_match_finite_differences():
    g = np.random.default_rng(0)
    din, dh, dout, B = 6, 5, 4, 7
    params = [g.normal(size=(dh, din)) * 0.5, g.normal(size=dh) * 0.1,
              g.normal(size=(dh, dh)) * 0.5, g.normal(size=dh) * 0.1,
              g.normal(size=(dout, dh)) * 0.5, g.normal(size=dout) * 0.1]
    X = g.normal(size=(B, din))
    T = g.normal(size=(B, dout))
    loss, grads = mlp.loss_grad(params, X, T)
    h = 1e-6
    for p, gp in zip(params, grads):
        flat = p.reshape(-1)
        gflat = gp.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp, _ = mlp.loss_grad(params, X, T)
            flat[i] = old - h
            lm, _ = mlp.loss_grad(params, X, T)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (fd, gflat[i])


def test_loss_is_sign_invariant_in_the_null_vector():
    g = np.random.default_rng(1)
    Y = g.normal(size=(3, 5))
    T = g.normal(size=(3, 5))
    l1, _ = mlp.loss_and_grad_out(Y, T)
    T2 = T.copy()
    T2[:, 1:] *= -1.0
    l2, _ = mlp.loss_and_grad_out(Y, T2)
    assert abs(l1 - l2) < 1e-14
