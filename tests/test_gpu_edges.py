"""Edge cases of the CUDA path against the FP64 oracle: an empty batch, and a
batch mixing an unglued subdomain (m = 0), exact tile multiples (m = 64,
32), a single multiplier (m = 1) and ragged sizes, through assembly, both
explicit applications and the implicit application."""
import numpy as np
import pytest

import oracle
from paper_2509_21037_gb300 import abi, host, implicit, sc

from test_abi import edge_batch

pytestmark = pytest.mark.gpu
TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_empty_batch(dev):
    plan = sc.Plan([], 0).upload(dev)
    F = plan.new_F(dev)
    Lv = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.assemble(Lv, F)
    assert plan.device_status() == abi.SC_OK
    lam = torch.zeros(1, dtype=torch.float64, device=dev)
    q = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.apply(F, lam, q)
    plan.apply_fixed(F, lam, q)
    torch.cuda.synchronize()


def test_edge_batch(dev):
    prob = edge_batch()
    fs = host.factorize_problem(prob.subdomains)
    assert [f.m for f in fs[:4]] == [0, 64, 32, 1]
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F = plan.new_F(dev)
    F.fill_(float("nan"))
    plan.assemble(Lv, F)
    assert plan.device_status() == abi.SC_OK
    assert plan.F_offsets[1] == plan.F_offsets[0]          # the unglued subdomain owns no F
    assert torch.isfinite(F).all()
    Fo = [np.zeros((0, 0))] + oracle.dual_operators(prob.subdomains[1:])
    for i in range(1, len(fs)):
        assert oracle.relative_frobenius(plan.export(F, i).cpu().numpy(), Fo[i]) <= TOL
    lam = torch.from_numpy(np.random.default_rng(4).standard_normal(prob.n_dual)).to(dev)
    qo = oracle.apply_dual(Fo, [s.lambda_map for s in prob.subdomains], lam.cpu().numpy(), prob.n_dual)
    for fn in (plan.apply, plan.apply_fixed):
        q = torch.empty_like(lam)
        fn(F, lam, q)
        assert np.linalg.norm(q.cpu().numpy() - qo) <= TOL * np.linalg.norm(qo)
    ip = implicit.ImplicitPlan(fs, prob.n_dual).upload(dev)
    q = torch.empty_like(lam)
    ip.apply(Lv, lam, q)
    assert ip.device_status() == abi.SC_OK
    assert np.linalg.norm(q.cpu().numpy() - qo) <= TOL * np.linalg.norm(qo)
