"""GPU parity of sc_apply_fixed (include/sc.h): F * lambda with per-tile
53-bit fixed point and exact integer multiply-adds.  Against the oracle's
sum_i F_i lambda_i (1e-12, the FP64 path's bound) and against the FP64
sc_apply on the same F (1e-14: both round at the FP64 level)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from paper_2509_21037_gb300 import abi, host, sc

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


def _q(plan, F, lam, dev, fixed=True):
    lam_d = torch.from_numpy(lam).to(dev)
    q = torch.full_like(lam_d, float("nan"))
    (plan.apply_fixed if fixed else plan.apply)(F, lam_d, q)
    return q.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,prob", [("config1", synth.make_config(1)), ("cube_coef", synth.cube_heat_3d(2, 6, coef_seed=3)),
                                       ("elast", synth.elasticity_cubes((2, 2, 1), 3, 6, seed=2)),
                                       ("mixed", synth.mixed_batch(lat2d=(2, 2), k2d=(6, 40), lat3d=(2, 1, 1), k3d=(2, 5), seed=1))],
                         ids=lambda x: x if isinstance(x, str) else "")
def test_apply_fixed_matches_oracle_and_fp64(name, prob, dev):
    plan, F = _setup(prob, dev)
    lam = np.random.default_rng(2).standard_normal(prob.n_dual)
    qf, q64 = _q(plan, F, lam, dev), _q(plan, F, lam, dev, fixed=False)
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains, refine=1), [s.lambda_map for s in prob.subdomains],
                           lam, prob.n_dual)
    print(f"{name}: fixed vs oracle {_rel(qf, qo):.2e}, vs FP64 apply {_rel(qf, q64):.2e}")
    assert _rel(qf, qo) <= 1e-12 and _rel(qf, q64) <= 1e-14


def test_apply_fixed_config2_and_dynamic_range(dev):
    """Config 2; lambda spanning 1e-150 .. 1e150 and an all-zero block; F
    scaled by 2^-700 and 2^+700 (the exponent scaling leaves the normal range
    on the way)."""
    prob = synth.make_config(2)
    plan, F = _setup(prob, dev)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(prob.n_dual)
    q64 = _q(plan, F, lam, dev, fixed=False)
    assert _rel(_q(plan, F, lam, dev), q64) <= 1e-14
    wild = lam * 10.0 ** rng.uniform(-150, 150, prob.n_dual)
    wild[:64] = 0.0
    assert _rel(_q(plan, F, wild, dev), _q(plan, F, wild, dev, fixed=False)) <= 1e-13
    for s in (2.0 ** -700, 2.0 ** 700):
        Fs = F * s
        # undo the power-of-two scale before the norms (their squares would leave the FP64 range)
        assert _rel(_q(plan, Fs, lam, dev) / s, q64) <= 1e-14
    assert np.all(_q(plan, F, np.zeros(prob.n_dual), dev) == 0.0)


@pytest.mark.parametrize("quarters", [0, 1, 2, 3, 4])
def test_apply_mixed_every_split(quarters, dev):
    """sc_apply_mixed: of every four tiles `quarters` run on the FP64 pipe and
    the rest in fixed point.  Against the oracle (1e-12) and the FP64 apply
    (1e-14) for every split, on a mixed batch whose subdomains have 1..many
    tile columns; quarters = 0 is sc_apply_fixed (the same kernel; q's
    atomic accumulation order differs run to run, so to rounding)."""
    prob = synth.mixed_batch(lat2d=(2, 2), k2d=(6, 40), lat3d=(2, 1, 1), k3d=(2, 5), seed=1)
    plan, F = _setup(prob, dev)
    lam = np.random.default_rng(3).standard_normal(prob.n_dual)
    lam_d = torch.from_numpy(lam).to(dev)
    q = torch.full_like(lam_d, float("nan"))
    plan.apply_mixed(F, lam_d, q, quarters)
    qm = q.cpu().numpy()
    q64 = _q(plan, F, lam, dev, fixed=False)
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains, refine=1), [s.lambda_map for s in prob.subdomains],
                           lam, prob.n_dual)
    assert _rel(qm, qo) <= 1e-12 and _rel(qm, q64) <= 1e-14
    if quarters == 0:
        assert _rel(qm, _q(plan, F, lam, dev)) <= 1e-15
    with pytest.raises(sc.SCError):
        plan.apply_mixed(F, lam_d, q, 5)
