"""GPU MLP kernels against the FP64 CPU reference (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp as om

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("B", [1, 37, 1000])
def test_forward_and_gradient_match_cpu_reference(dev, B):
    from paper_2509_21037_gb300.mlp import MLP
    rng = np.random.default_rng(B)
    net = MLP(12, 64, 10, device=dev, seed=B)
    X = rng.standard_normal((B, 12)).astype(np.float32)
    T = rng.standard_normal((B, 10)).astype(np.float32)
    M = (rng.random((B, 10)) > 0.3).astype(np.float32)
    M[0, 0] = 1.0
    Xd, Td, Md = (torch.from_numpy(a).to(dev) for a in (X, T, M))
    p = net.params.cpu().numpy().astype(np.float64)
    y_ref, _ = om.forward(p, X, (12, 64, 10))
    y = net.forward(Xd).cpu().numpy()
    assert np.max(np.abs(y - y_ref)) <= 1e-4 * max(1.0, np.abs(y_ref).max())
    loss = net.loss_grad(Xd, Td, Md)
    L_ref, g_ref = om.loss_grad(p, X, T, M, (12, 64, 10))
    assert abs(float(loss.item()) - L_ref) <= 1e-4 * max(1.0, L_ref)
    g = net.grads.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_training_fits_a_smooth_target(dev):
    from paper_2509_21037_gb300.mlp import MLP
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (512, 6))
    T = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] ** 2, X[:, 2] * X[:, 3]], axis=1)
    net = MLP(6, 64, 2, device=dev, seed=1)
    hist = net.fit(X, T, np.ones_like(T), epochs=1500, lr=3e-3)
    assert hist[-1] < 0.05 * hist[0]
    pred = net.predict(X)
    assert np.mean((pred - T) ** 2) < 0.01
