"""GPU parity of the tensor-core apply from the digit form of F
(include/sc.h: sc_apply_digits_prepare, sc_apply_digits): against the
oracle's sum_i F_i lambda_i (1e-12, the FP64 path's bound) and against the
FP64 sc_apply on the same F (1e-14: both round at the FP64 level), on batches
whose subdomains have one to many tile columns, empty and ragged
subdomains, config 2, lambda of wide dynamic range and F scaled out of the
normal exponent range on the way."""
import numpy as np
import pytest

import oracle
import synth
from paper_2509_21037_gb300 import abi, host, sc
from test_abi import edge_batch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _setup(prob, dev):
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    F = plan.new_F(dev)
    plan.assemble(torch.from_numpy(sc.concat_L_values(fs)).to(dev), F)
    assert plan.device_status() == abi.SC_OK
    return plan, F


def _q(plan, F, lam, dev, Fd=None):
    lam_d = torch.from_numpy(lam).to(dev)
    q = torch.full_like(lam_d, float("nan"))
    if Fd is None:
        plan.apply(F, lam_d, q)
    else:
        plan.apply_digits(Fd, lam_d, q)
    return q.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,prob", [("config1", synth.make_config(1)), ("edge_batch", edge_batch()),
                                       ("cube_coef", synth.cube_heat_3d(2, 6, coef_seed=3)),
                                       ("elast", synth.elasticity_cubes((2, 2, 1), 3, 6, seed=2)),
                                       ("mixed", synth.mixed_batch(lat2d=(2, 2), k2d=(6, 40), lat3d=(2, 1, 1), k3d=(2, 5), seed=1))],
                         ids=lambda x: x if isinstance(x, str) else "")
def test_apply_digits_matches_oracle_and_fp64(name, prob, dev):
    plan, F = _setup(prob, dev)
    Fd = plan.prepare_digits(F)
    ntiles = plan.sizes.F_doubles // 1024
    assert plan.digits_size() == ntiles * 7184 + sum(-(-m // 32) for m in plan.m) * 944 + 16
    lam = np.random.default_rng(2).standard_normal(prob.n_dual)
    qd, q64 = _q(plan, F, lam, dev, Fd), _q(plan, F, lam, dev)
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains, refine=1), [s.lambda_map for s in prob.subdomains],
                           lam, prob.n_dual)
    print(f"{name}: digits vs oracle {_rel(qd, qo):.2e}, vs FP64 apply {_rel(qd, q64):.2e}")
    assert _rel(qd, qo) <= 1e-12 and _rel(qd, q64) <= 1e-14
    # unglued multipliers of the batch get exactly zero, as from the FP64 apply
    assert np.array_equal(qd == 0.0, q64 == 0.0)
    assert plan.digits_status(Fd) == abi.SC_OK


def test_apply_digits_config2_and_dynamic_range(dev):
    """Config 2; lambda spanning 1e-150 .. 1e150 and an all-zero block; F
    scaled by 2^-700 and 2^+700; a second call on the same digit form (the
    per-call lambda scratch is rewritten) and lambda = 0."""
    prob = synth.make_config(2)
    plan, F = _setup(prob, dev)
    Fd = plan.prepare_digits(F)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(prob.n_dual)
    q64 = _q(plan, F, lam, dev)
    r = _rel(_q(plan, F, lam, dev, Fd), q64)
    print(f"config 2: digits vs FP64 apply {r:.2e}")
    assert r <= 1e-14
    wild = lam * 10.0 ** rng.uniform(-150, 150, prob.n_dual)
    wild[:64] = 0.0
    assert _rel(_q(plan, F, wild, dev, Fd), _q(plan, F, wild, dev)) <= 1e-13
    assert _rel(_q(plan, F, lam, dev, Fd), q64) <= 1e-14
    for s in (2.0 ** -700, 2.0 ** 700):
        Fs = F * s
        Fds = plan.prepare_digits(Fs)
        assert _rel(_q(plan, Fs, lam, dev, Fds) / s, q64) <= 1e-14
    assert np.all(_q(plan, F, np.zeros(prob.n_dual), dev, Fd) == 0.0)


def test_apply_digits_rejects_misaligned_buffer(dev):
    plan, F = _setup(synth.make_config(1), dev)
    Fd = torch.empty(plan.digits_size() + 16, dtype=torch.uint8, device=dev)
    with pytest.raises(sc.SCError):
        plan.prepare_digits(F, Fd[1:])


def test_apply_digits_bounded_waits(dev):
    """poll_limit = 1: the product kernel's waits for its bulk copies may give
    up; it then reports SC_ERR_TIMEOUT through the status word (never a
    fault), and the context stays usable: a plan with the default bound gives
    the FP64 product."""
    prob = synth.make_config(1)
    fs = host.factorize_problem(prob.subdomains)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    lam = np.random.default_rng(7).standard_normal(prob.n_dual)
    tight = sc.Plan(fs, prob.n_dual, poll_limit=1).upload(dev)
    F = tight.new_F(dev)
    tight.assemble(Lv, F)
    Fd = tight.prepare_digits(F)
    _q(tight, F, lam, dev, Fd)
    st = tight.digits_status(Fd)
    assert st in (abi.SC_OK, abi.SC_ERR_TIMEOUT)
    print(f"poll_limit = 1: status {st}")
    plan, F2 = _setup(prob, dev)
    Fd2 = plan.prepare_digits(F2)
    assert _rel(_q(plan, F2, lam, dev, Fd2), _q(plan, F2, lam, dev)) <= 1e-14
    assert plan.digits_status(Fd2) == abi.SC_OK
