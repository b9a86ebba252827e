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


def test_adam_kernel_matches_fp64_reference(dev):
    """sc_mlp_adam (FP32 on the GPU) against oracle.mlp.adam_step (FP64),
    element by element over 12 steps of a seeded gradient sequence, with the
    bias correction active (steps 1..12 of beta2 = 0.999 leave 1 - beta2^t far
    from 1).  The oracle gets the hyperparameters the kernel receives (their
    FP32 values), so only FP32 arithmetic separates the two.  Tolerances from
    that arithmetic: each step adds a few FP32 roundings relative to the
    largest gradient seen so far (m is a weighted mean of the g's and v of the
    g^2's, so cancellation in m can leave the error of an earlier, larger g),
    at most t 2^-21 max|g| (resp. max g^2) after t steps;
    the step's bias corrections 1 - beta^t lose up to 2^-23 / (1 - beta2^t)
    ~ 2^-17 to cancellation, so each update is good to lr 2^-12 at most,
    and the stored params round by 2^-24 |p| per step."""
    import ctypes
    from paper_2509_21037_gb300.mlp import _lib
    lib = _lib()
    rng = np.random.default_rng(5)
    n, K = 4099, 12                                # ragged against the 256-thread blocks
    f32 = lambda x: float(np.float32(x))
    lr, b1, b2, eps = f32(3e-3), f32(0.9), f32(0.999), f32(1e-8)
    p0 = rng.standard_normal(n).astype(np.float32)
    gs = [(rng.standard_normal(n) * np.exp(rng.uniform(-6, 3, n))).astype(np.float32) for _ in range(K)]
    gs[0][:7] = 0.0                                # zero gradients: v = 0 there, eps guards the division
    p = torch.from_numpy(p0.copy()).to(dev)
    m = torch.zeros(n, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    pr, mr, vr = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    moved = np.zeros(n)
    gmax = np.zeros(n)                             # running max |g|: the scale of every m (a weighted mean of g)
    for t in range(1, K + 1):
        g64 = gs[t - 1].astype(np.float64)
        gmax = np.maximum(gmax, np.abs(g64))
        g = torch.from_numpy(gs[t - 1]).to(dev)
        rc = lib.sc_mlp_adam(n, p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), ctypes.c_float(lr),
                             ctypes.c_float(b1), ctypes.c_float(b2), ctypes.c_float(eps), t, None)
        assert rc == 0
        pn, mr, vr = om.adam_step(pr, g64, mr, vr, lr, b1, b2, eps, t)
        moved += np.abs(pn - pr)
        pr = pn
        pg, mg, vg = (x.cpu().numpy().astype(np.float64) for x in (p, m, v))
        assert np.all(np.abs(mg - mr) <= t * 2.0 ** -21 * gmax), f"m at step {t}"
        assert np.all(np.abs(vg - vr) <= t * 2.0 ** -21 * gmax ** 2), f"v at step {t}"
        assert np.all(np.abs(pg - pr) <= t * (2.0 ** -23 * np.abs(pr) + lr * 2.0 ** -12)), f"params at step {t}"
    # the updates are large against the tolerance (the comparison is not vacuous)
    assert np.median(moved) > 100 * K * lr * 2.0 ** -12
