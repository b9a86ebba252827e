"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative Frobenius error ||F_gpu - F_oracle||_F / ||F_oracle||_F
<= 1e-12 per subdomain (FP64 path), and the same bound on ||q - q_oracle|| /
||q_oracle|| for the explicit application.
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from paper_2509_21037_gb300 import abi, host, sc

pytestmark = pytest.mark.gpu
TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _assemble(prob_or_fs, n_dual, dev, subdomains=None):
    fs = prob_or_fs
    plan = sc.Plan(fs, n_dual).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F = plan.new_F(dev)
    F.fill_(float("nan"))               # every entry must be written by the library
    plan.assemble(Lv, F)
    assert plan.device_status() == abi.SC_OK
    return plan, F, Lv


def _check_all(plan, F, Fo, tol=TOL):
    worst = 0.0
    for i in range(plan.nsub):
        Fg = plan.export(F, i).cpu().numpy()
        assert np.isfinite(Fg).all()
        worst = max(worst, oracle.relative_frobenius(Fg, Fo[i]))
    assert worst <= tol, f"max relative Frobenius error {worst:.3e}"
    return worst


def _padding_zero(plan, F):
    Fh = F.cpu().numpy()
    assert np.isfinite(Fh).all(), "unwritten (NaN) entries in the F buffer"
    for i in range(plan.nsub):
        m = plan.m[i]
        nt = (m + 31) // 32
        if nt == 0 or m % 32 == 0:
            continue
        I = nt - 1
        for J in range(I + 1):
            T = Fh[plan.F_offsets[i] + (I * (I + 1) // 2 + J) * 1024:][:1024].reshape(32, 32).T  # [row, col]
            assert np.all(T[m - 32 * I:, :] == 0)
            if J == I:
                assert np.all(T[:, m - 32 * I:] == 0)


def test_config1(dev):
    prob = synth.make_config(1)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, _ = _assemble(fs, prob.n_dual, dev)
    Fo = oracle.dual_operators(prob.subdomains)
    _check_all(plan, F, Fo)
    _padding_zero(plan, F)
    Fg = plan.export(F, 0).cpu().numpy()
    assert np.array_equal(Fg, Fg.T)


@pytest.mark.parametrize("k", [3, 6, 9])
def test_small_cubes_ragged(dev, k):
    prob = synth.cube_heat_3d(parts=2, k=k)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, _ = _assemble(fs, prob.n_dual, dev)
    _check_all(plan, F, oracle.dual_operators(prob.subdomains))
    _padding_zero(plan, F)


def test_random_coefficients_no_dedup(dev):
    """Per-subdomain conductivities: every subdomain's L values differ, so a
    path that reused one subdomain's numbers for another would fail."""
    prob = synth.cube_heat_3d(parts=2, k=6, coef_seed=11)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, _ = _assemble(fs, prob.n_dual, dev)
    _check_all(plan, F, oracle.dual_operators(prob.subdomains))


def test_elasticity_uneven(dev):
    prob = synth.elasticity_cubes((2, 2, 1), 3, 6, seed=2)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, _ = _assemble(fs, prob.n_dual, dev)
    _check_all(plan, F, oracle.dual_operators(prob.subdomains, refine=1))


def test_general_gluing_columns(dev):
    """B^T columns with several nonzeros, an empty column, duplicate dofs."""
    base = synth.cube_heat_3d(parts=1, k=5).subdomains[0]
    rng = np.random.default_rng(7)
    n, m = base.n, 75
    rows, cols, vals = [], [], []
    for j in range(m):
        if j == 40:
            continue                                  # empty column
        k = 3 if j % 7 == 0 else 1
        for r in rng.choice(n, size=k, replace=False):
            rows.append(r); cols.append(j); vals.append(rng.choice([-1.0, 1.0]))
    Bt = sp.csc_matrix((vals, (rows, cols)), shape=(n, m))
    sd = synth.Subdomain(K=base.K, fixed=base.fixed, Bt=Bt, lambda_map=np.arange(m), grid=base.grid,
                         ndpn=1, key=None)
    fs = host.factorize_problem([sd])
    plan, F, _ = _assemble(fs, m, dev)
    _check_all(plan, F, [oracle.dual_operator(sd)])


def test_config2_full(dev):
    prob = synth.make_config(2)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, _ = _assemble(fs, prob.n_dual, dev)
    Fo = oracle.dual_operators(prob.subdomains, refine=1)
    worst = _check_all(plan, F, Fo)
    print(f"config 2: max relative Frobenius error vs refined oracle {worst:.3e}")
    _padding_zero(plan, F)
    # explicit application, whole dual vector
    lam = torch.from_numpy(np.random.default_rng(2).standard_normal(prob.n_dual)).to(dev)
    q = torch.full_like(lam, float("nan"))
    plan.apply(F, lam, q)
    qo = oracle.apply_dual(Fo, [s.lambda_map for s in prob.subdomains], lam.cpu().numpy(), prob.n_dual)
    err = np.linalg.norm(q.cpu().numpy() - qo) / np.linalg.norm(qo)
    assert err <= TOL


def test_apply_small(dev):
    prob = synth.cube_heat_3d(parts=2, k=7)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, _ = _assemble(fs, prob.n_dual, dev)
    Fo = oracle.dual_operators(prob.subdomains)
    for seed in range(3):
        lam = torch.from_numpy(np.random.default_rng(seed).standard_normal(prob.n_dual)).to(dev)
        q = torch.empty_like(lam)
        plan.apply(F, lam, q)
        qo = oracle.apply_dual(Fo, [s.lambda_map for s in prob.subdomains], lam.cpu().numpy(), prob.n_dual)
        assert np.linalg.norm(q.cpu().numpy() - qo) <= TOL * np.linalg.norm(qo)


def test_repeat_is_bitwise_deterministic_and_values_reuse(dev):
    prob = synth.cube_heat_3d(parts=2, k=5)
    fs = host.factorize_problem(prob.subdomains)
    plan, F, Lv = _assemble(fs, prob.n_dual, dev)
    F2 = plan.new_F(dev)
    plan.assemble(Lv, F2)
    assert torch.equal(F, F2)
    # new numeric values, same pattern (paper Sec. 2.2: symbolic stage reused):
    # L -> 2 L gives K -> 4 K and F -> F / 4 exactly (powers of two)
    plan.assemble(Lv * 2.0, F2)
    assert plan.device_status() == abi.SC_OK
    assert torch.equal(F2 * 4.0, F)


def test_not_spd_reported(dev):
    prob = synth.cube_heat_3d(parts=2, k=4)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    Lv = sc.concat_L_values(fs).copy()
    # negate the diagonal of the last column of subdomain 3 (a root: always active)
    c = fs[3].n - 1
    Lv[plan.L_offsets[3] + fs[3].L.colptr[c]] *= -1.0
    F = plan.new_F(dev)
    plan.assemble(torch.from_numpy(Lv).to(dev), F)
    assert plan.device_status() == abi.SC_ERR_NOT_SPD
    # the context stays usable
    plan.assemble(torch.from_numpy(sc.concat_L_values(fs)).to(dev), F)
    assert plan.device_status() == abi.SC_OK


def test_workspace_too_small_rejected(dev):
    prob = synth.make_config(1)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F = plan.new_F(dev)
    small = torch.empty(plan.sizes.ws_bytes // 2, dtype=torch.uint8, device=dev)
    with pytest.raises(sc.SCError) as e:
        plan.assemble(Lv, F, ws=small)
    assert e.value.status == abi.SC_ERR_OOM


def test_dense_comparator_matches_oracle(dev):
    from paper_2509_21037_gb300 import dense
    prob = synth.make_config(1)
    fs = host.factorize_problem(prob.subdomains)
    Fd = dense.assemble_dense(fs, dev, emulation=0)
    Fo = oracle.dual_operators(prob.subdomains)
    assert oracle.relative_frobenius(Fd[0], Fo[0]) <= TOL


def test_cuda_graph_capture_replay(dev):
    """sc_assemble_batch + sc_apply captured in one CUDA graph and replayed."""
    prob = synth.cube_heat_3d(parts=2, k=6, coef_seed=1)
    fs = host.factorize_problem(prob.subdomains)
    plan, F_ref, Lv = _assemble(fs, prob.n_dual, dev)
    lam = torch.from_numpy(np.random.default_rng(4).standard_normal(prob.n_dual)).to(dev)
    q_ref = torch.empty_like(lam)
    plan.apply(F_ref, lam, q_ref)
    F = plan.new_F(dev)
    q = torch.empty_like(lam)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.assemble(Lv, F, stream=s)
            plan.apply(F, lam, q, stream=s)
    for _ in range(3):
        F.fill_(float("nan"))
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(F, F_ref)
    assert torch.allclose(q, q_ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("split", [0, 5])
def test_workspace_waves_match_single_wave(dev, split):
    """A workspace bound splits the batch into waves reusing one workspace;
    the result equals the single-wave assembly bit for bit."""
    prob = synth.cube_heat_3d(parts=2, k=6, coef_seed=2)
    fs = host.factorize_problem(prob.subdomains)
    var = [split] * len(fs)
    ref_plan, F_ref, Lv = None, None, None
    ref_plan = sc.Plan(fs, prob.n_dual, sub_slices=var).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F_ref = ref_plan.new_F(dev)
    ref_plan.assemble(Lv, F_ref)
    plan = sc.Plan(fs, prob.n_dual, sub_slices=var, ws_limit=ref_plan.sizes.ws_bytes // 3).upload(dev)
    assert plan.stats.n_waves >= 3
    F = plan.new_F(dev)
    F.fill_(float("nan"))
    plan.assemble(Lv, F)
    assert plan.device_status() == abi.SC_OK
    assert torch.equal(F, F_ref)


@pytest.mark.parametrize("name", ["config2", "mixed_waves"])
def test_persistent_work_queue_bitwise(name, dev):
    """sc_options.persistent: resident CTAs pulling tasks from an atomic
    counter compute exactly what one CTA per task computes."""
    if name == "config2":
        prob = synth.make_config(2)
        kw = {}
    else:
        prob = synth.mixed_batch(lat2d=(2, 2), k2d=(6, 40), lat3d=(2, 1, 1), k3d=(2, 6), seed=3)
        kw = {}
    fs = host.factorize_problem(prob.subdomains)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    out = []
    for pers in (False, True):
        one = sc.Plan(fs, prob.n_dual).upload(dev)
        lim = one.sizes.ws_bytes // 2 if name == "mixed_waves" else 0
        plan = sc.Plan(fs, prob.n_dual, ws_limit=lim, persistent=pers).upload(dev)
        F = plan.new_F(dev)
        F.fill_(float("nan"))
        plan.assemble(Lv, F)
        assert plan.device_status() == abi.SC_OK
        out.append(F.cpu().numpy())
    assert np.array_equal(out[0], out[1])
