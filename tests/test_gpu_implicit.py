"""GPU parity of the implicit dual-operator application (include/sc_implicit.h):
q = sum_i B_i L_i^{-T} L_i^{-1} B_i^T lambda_i against the FP64 oracle's
sum_i F_i lambda_i, and against the explicit sc_apply on the assembled F.

Tolerance: ||q_gpu - q_oracle|| <= 1e-12 ||q_oracle|| (FP64 path).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from paper_2509_21037_gb300 import abi, host, implicit, sc

pytestmark = pytest.mark.gpu
TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _implicit_q(fs, n_dual, lam, dev, cluster_min_work=-1, pairs=0):
    ip = implicit.ImplicitPlan(fs, n_dual, cluster_min_work=cluster_min_work, pairs=pairs).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    lam_d = torch.from_numpy(lam).to(dev)
    q = torch.full((max(1, n_dual),), float("nan"), dtype=torch.float64, device=dev)
    ip.apply(Lv, lam_d, q)
    assert ip.device_status() == abi.SC_OK
    return ip, q[:n_dual].cpu().numpy()


def _oracle_q(subs, lam, n_dual, refine=0):
    return oracle.apply_dual(oracle.dual_operators(subs, refine=refine), [s.lambda_map for s in subs], lam, n_dual)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cases():
    yield "config1", synth.make_config(1)
    yield "cube_2x8", synth.cube_heat_3d(2, 8)
    yield "cube_coef", synth.cube_heat_3d(2, 6, coef_seed=3)
    yield "elast", synth.elasticity_cubes((2, 2, 1), 3, 6, seed=2)
    yield "mixed", synth.mixed_batch(lat2d=(2, 2), k2d=(6, 40), lat3d=(2, 1, 1), k3d=(2, 5), seed=1)


@pytest.mark.parametrize("name,prob", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_implicit_matches_oracle(name, prob, dev):
    fs = host.factorize_problem(prob.subdomains)
    lam = np.random.default_rng(11).standard_normal(prob.n_dual)
    _, q = _implicit_q(fs, prob.n_dual, lam, dev)
    err = _rel(q, _oracle_q(prob.subdomains, lam, prob.n_dual, refine=1))
    print(f"{name}: implicit apply vs oracle {err:.3e}")
    assert err <= TOL


@pytest.mark.parametrize("mode", ["all_clusters", "no_clusters", "mixed", "pairs", "mixed_pairs"])
def test_implicit_cluster_modes(mode, dev):
    """Every subdomain on an 8-CTA cluster, every subdomain on one CTA, a mix
    (large ones on clusters, small ones packed one per CTA), every subdomain
    on a CTA pair (its two subtrees solved side by side), and large ones on
    clusters with the rest on pairs: same q."""
    prob = synth.mixed_batch(lat2d=(4, 4), k2d=(6, 40), lat3d=(2, 2, 1), k3d=(2, 8), seed=2)
    fs = host.factorize_problem(prob.subdomains)
    nnz = implicit.ImplicitPlan(fs, prob.n_dual).sizes.nnz_visited
    cmw = {"all_clusters": 0, "no_clusters": 1 << 60, "mixed": nnz // 40, "pairs": 1 << 60,
           "mixed_pairs": nnz // 40}[mode]
    pairs = 1 if mode in ("pairs", "mixed_pairs") else -1
    lam = np.random.default_rng(4).standard_normal(prob.n_dual)
    ip, q = _implicit_q(fs, prob.n_dual, lam, dev, cmw, pairs)
    if mode.startswith("mixed"):
        assert 0 < ip.sizes.n_cluster_subdomains < len(fs)
    err = _rel(q, _oracle_q(prob.subdomains, lam, prob.n_dual, refine=1))
    print(f"cluster mode {mode}: {ip.sizes.n_cluster_subdomains} of {len(fs)} on clusters, error {err:.3e}")
    assert err <= TOL


def test_implicit_general_gluing(dev):
    """B^T columns with several nonzeros, an empty column and a shared dof."""
    base = synth.cube_heat_3d(parts=1, k=6).subdomains[0]
    rng = np.random.default_rng(7)
    n, m = base.n, 70
    rows, cols, vals = [], [], []
    for j in range(m):
        if j == 33:
            continue
        k = 3 if j % 5 == 0 else 1
        for r in rng.choice(n, size=k, replace=False):
            rows.append(r); cols.append(j); vals.append(rng.choice([-1.0, 1.0]))
    rows.append(rows[0]); cols.append(m - 1); vals.append(-1.0)
    Bt = sp.csc_matrix((vals, (rows, cols)), shape=(n, m))
    sd = synth.Subdomain(K=base.K, fixed=base.fixed, Bt=Bt, lambda_map=np.arange(m), grid=base.grid, ndpn=1,
                         key=None)
    fs = host.factorize_problem([sd])
    lam = rng.standard_normal(m)
    _, q = _implicit_q(fs, m, lam, dev)
    assert _rel(q, _oracle_q([sd], lam, m)) <= TOL


def test_implicit_equals_explicit_config2(dev):
    """Config 2 (64 subdomains of 4913 dofs): the implicit and the explicit
    application of the same operator agree, and both match the oracle."""
    prob = synth.make_config(2)
    fs = host.factorize_problem(prob.subdomains)
    lam = np.random.default_rng(3).standard_normal(prob.n_dual)
    ip, qi = _implicit_q(fs, prob.n_dual, lam, dev)
    _, qs = _implicit_q(fs, prob.n_dual, lam, dev, pairs=-1)     # one CTA per subdomain
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F = plan.new_F(dev)
    plan.assemble(Lv, F)
    q = torch.empty(prob.n_dual, dtype=torch.float64, device=dev)
    plan.apply(F, torch.from_numpy(lam).to(dev), q)
    qe = q.cpu().numpy()
    memo = oracle._Memo()
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains, memo, refine=1),
                           [s.lambda_map for s in prob.subdomains], lam, prob.n_dual)
    e_imp, e_exp, e_ie = _rel(qi, qo), _rel(qe, qo), _rel(qi, qe)
    print(f"config 2: implicit {e_imp:.3e}, explicit {e_exp:.3e}, implicit vs explicit {e_ie:.3e}, "
          f"CTA pairs vs one CTA {_rel(qi, qs):.3e}")
    assert e_imp <= TOL and e_exp <= TOL and e_ie <= TOL and _rel(qi, qs) <= TOL


def test_implicit_repeatable_and_reusable(dev):
    """Repeated calls with new values of lambda and of L (same patterns) reuse
    the plan; results are reproducible up to the order of atomic additions."""
    prob = synth.cube_heat_3d(2, 7, coef_seed=5)
    fs = host.factorize_problem(prob.subdomains)
    ip = implicit.ImplicitPlan(fs, prob.n_dual).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    rng = np.random.default_rng(1)
    for _ in range(3):
        lam = rng.standard_normal(prob.n_dual)
        q = torch.empty(prob.n_dual, dtype=torch.float64, device=dev)
        ip.apply(Lv, torch.from_numpy(lam).to(dev), q)
        assert _rel(q.cpu().numpy(), _oracle_q(prob.subdomains, lam, prob.n_dual)) <= TOL
    # L scaled by c: K scaled by c^2, so q scales by 1 / c^2
    q1 = torch.empty(prob.n_dual, dtype=torch.float64, device=dev)
    ip.apply(Lv * 4.0, torch.from_numpy(lam).to(dev), q1)
    assert _rel(q1.cpu().numpy() * 16.0, q.cpu().numpy()) <= 1e-14


def test_implicit_not_spd_is_reported(dev):
    prob = synth.cube_heat_3d(2, 4)
    fs = host.factorize_problem(prob.subdomains)
    ip = implicit.ImplicitPlan(fs, prob.n_dual).upload(dev)
    vals = sc.concat_L_values(fs).copy()
    vals[fs[0].L.colptr[fs[0].n - 1]] = -1.0           # L_0's last diagonal entry (the etree root, always visited)
    q = torch.empty(prob.n_dual, dtype=torch.float64, device=dev)
    ip.apply(torch.from_numpy(vals).to(dev), torch.ones(prob.n_dual, dtype=torch.float64, device=dev), q)
    assert ip.device_status() == abi.SC_ERR_NOT_SPD


def test_implicit_workspace_checks(dev):
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    ip = implicit.ImplicitPlan(fs, prob.n_dual).upload(dev)
    ip.ws = ip.ws[:ip.sizes.ws_bytes // 2]
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    q = torch.empty(prob.n_dual, dtype=torch.float64, device=dev)
    with pytest.raises(sc.SCError, match="SC_ERR_OOM"):
        ip.apply(Lv, torch.ones(prob.n_dual, dtype=torch.float64, device=dev), q)


def test_implicit_large_batch_two_ctas_per_sm(dev):
    """More subdomains than SMs (176 on 152): the launch takes 8 warps and two
    CTAs per SM; q still matches the oracle."""
    prob = synth.mixed_batch(lat2d=(14, 12), k2d=(4, 10), lat3d=(2, 2, 2), k3d=(2, 4), seed=5)
    assert len(prob.subdomains) > 152
    fs = host.factorize_problem(prob.subdomains)
    lam = np.random.default_rng(8).standard_normal(prob.n_dual)
    _, q = _implicit_q(fs, prob.n_dual, lam, dev)
    err = _rel(q, _oracle_q(prob.subdomains, lam, prob.n_dual, refine=1))
    print(f"{len(fs)} subdomains: implicit apply vs oracle {err:.3e}")
    assert err <= TOL
