"""The warm-start network's GPU kernels (tcgen05 BF16 GEMMs, FP32
accumulation) against the FP64 CPU reference (oracle/mlp.py).

The GPU rounds inputs, weights and activations to BF16 (8 significant bits),
so the comparison is made on the same BF16-rounded parameters and inputs and
allows the BF16 rounding of the activations: outputs within 3e-2 of the
output scale, the gradient vector within cosine 0.995 and a relative norm
error of 5e-2 per layer."""
import numpy as np
import pytest

from oracle import mlp as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spectra():
    from paper_2010_03817_gb300 import build, spectra as S
    build.build()
    return S


def _bf16(a):
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def _ref_rounded(params, X, T):
    """FP64 reference with the GPU's BF16 roundings of activations and of the
    back-propagated gradients (inputs of the tensor-core GEMMs)."""
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1.T + b1
    H1 = _bf16(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = _bf16(np.maximum(Z2, 0.0))
    Y = H2 @ W3.T + b3
    loss, dY = ref.loss_and_grad_out(Y, T)
    dY = _bf16(dY)
    gW3, gb3 = dY.T @ H2, dY.sum(0)
    dZ2 = _bf16(dY @ W3) * (H2 > 0)
    gW2, gb2 = dZ2.T @ H1, dZ2.sum(0)
    dZ1 = _bf16(dZ2 @ W2) * (H1 > 0)
    gW1, gb1 = dZ1.T @ X, dZ1.sum(0)
    return Y, loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def test_forward_and_gradients_match_reference(spectra):
    din, dh, dout, B = 37, 64, 21, 64
    net = spectra.MLP(din, dh, dout, seed=3)
    g = np.random.default_rng(4)
    X = g.normal(size=(B, din)).astype(np.float32)
    T = g.normal(size=(B, dout)).astype(np.float32)
    flat = net.params()
    W1, b1, W2, b2, W3, b3 = net.unflatten(flat)
    params = [_bf16(W1[:, :din]), b1.astype(np.float64), _bf16(W2), b2.astype(np.float64),
              _bf16(W3[:dout]), b3[:dout].astype(np.float64)]
    Xd = torch.tensor(X, device="cuda")
    Y = net.forward(Xd).cpu().numpy()
    Yr, _ = ref.forward(params, _bf16(X))
    assert np.abs(Y - Yr).max() <= 3e-2 * np.abs(Yr).max()
    loss, grad = net.gradients(Xd, torch.tensor(T, device="cuda"))
    Yq, lq, gq = _ref_rounded(params, _bf16(X), T.astype(np.float64))
    assert abs(loss - lq) <= 2e-2 * abs(lq), (loss, lq)
    gg = net.unflatten(grad)
    report = []
    for k, (a, b) in enumerate(zip(gg, gq)):
        a = a[:b.shape[0]] if a.ndim == 1 else a[:b.shape[0], :b.shape[1]]
        a, b = a.reshape(-1).astype(np.float64), b.reshape(-1)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        report.append((k, round(float(cos), 5), round(float(rel), 5)))
    assert all(c > 0.999 and r < 3e-2 for _, c, r in report), report
    # padded output rows of W3 get no gradient
    assert np.all(gg[4][dout:] == 0.0) and np.all(gg[5][dout:] == 0.0)


def test_training_reduces_the_loss(spectra):
    din, dh, dout, B = 16, 64, 9, 4096
    g = np.random.default_rng(5)
    X = g.normal(size=(B, din)).astype(np.float32)
    # a learnable target: log-length a linear function, null vector a fixed map of x
    T = np.empty((B, dout), dtype=np.float32)
    T[:, 0] = 0.5 * X[:, 0] - 0.25 * X[:, 1]
    M = g.normal(size=(dout - 1, din)).astype(np.float32)
    T[:, 1:] = X @ M.T
    net = spectra.MLP(din, dh, dout, seed=6)
    losses = net.train(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), epochs=60,
                       batch=256, lr=2e-3)
    assert losses[-1] < 0.3 * losses[0], losses


def test_save_and_load_round_trip(spectra, tmp_path):
    """sp_mlp_save / sp_mlp_load keep the dimensions, the parameters bit for
    bit and hence the forward pass."""
    net = spectra.MLP(20, 64, 22, seed=5)
    path = str(tmp_path / "net.spmlp")
    net.save(path)
    other = spectra.MLP.load(path)
    assert (other.din, other.dh, other.dout) == (20, 64, 22)
    assert np.array_equal(other.params(), net.params())
    X = torch.randn(64, 20, dtype=torch.float32, device="cuda")
    assert torch.equal(net.forward(X), other.forward(X))
    with open(path, "r+b") as f:  # a corrupted header is rejected
        f.write(b"XXXX")
    with pytest.raises(spectra.SpectraError):
        spectra.MLP.load(path)
