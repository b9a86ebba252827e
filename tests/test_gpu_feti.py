"""The FETI-1 PCPG solver (feti.py) on the library's assembled F: the dual
solution matches a projected CG on the oracle's operator, and the recovered
primal solution is continuous across the interface and in equilibrium."""
import numpy as np
import pytest

import synth
from paper_2509_21037_gb300 import feti

import test_feti as tf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


ITERATIONS = {}


@pytest.mark.parametrize("precond", ["none", "lumped", "dirichlet"])
def test_feti_solve_small_cube(precond, dev):
    prob = synth.cube_heat_3d(2, 4, coef_seed=3)
    loads = feti.compatible_loads(prob, seed=5)
    res = feti.FETISolver(prob, device=dev, precond=precond).solve(loads, tol=1e-12)
    F, G, d, e = tf._dual_problem(prob, loads)
    GtGp = np.linalg.pinv(G.T @ G, rcond=1e-12, hermitian=True)
    # the converged lambda solves the projected system: P (d - F lambda) = 0, G^T lambda = e
    r = d - F @ res.lam
    Pr = r - G @ (GtGp @ (G.T @ r))
    assert np.linalg.norm(Pr) <= 1e-9 * np.linalg.norm(d)
    assert np.allclose(G.T @ res.lam, e, atol=1e-10 * np.abs(e).max())
    assert res.continuity <= 1e-9 and res.equilibrium <= 1e-9
    print(f"{precond}: {res.iterations} iterations, continuity {res.continuity:.2e}, "
          f"equilibrium {res.equilibrium:.2e}")
    ITERATIONS[precond] = res.iterations
    if precond == "dirichlet" and {"none", "lumped"} <= ITERATIONS.keys():
        # the Dirichlet blocks go through the library's sc_apply on a tile-packed copy
        assert ITERATIONS["dirichlet"] < ITERATIONS["lumped"] < ITERATIONS["none"], ITERATIONS


def test_feti_solve_config2(dev):
    """Config 2 (64 floating subdomains): PCPG with the Dirichlet
    preconditioner converges; the primal solution is continuous and in
    equilibrium."""
    prob = synth.make_config(2)
    loads = feti.compatible_loads(prob, seed=1)
    res = feti.FETISolver(prob, device=dev, precond="dirichlet").solve(loads, tol=1e-10)
    print(f"config 2: {res.iterations} iterations, continuity {res.continuity:.2e}, equilibrium "
          f"{res.equilibrium:.2e}, F apply {res.apply_ms:.3f} ms, PCPG {res.solve_ms:.1f} ms")
    assert res.residuals[-1] < 1e-10
    assert res.continuity <= 1e-8 and res.equilibrium <= 1e-8


@pytest.mark.parametrize("name", ["cubes", "elasticity"])
def test_dirichlet_setup_on_the_gpu_matches_host(name, dev):
    """The Dirichlet preconditioner assembled on the GPU by the library
    (interior factors + general right-hand sides C_i = K_ib B_b^T, the
    library's own sc_assemble_batch) equals the dense host Schur complements
    block by block (1e-12), and the solves take the same iterations."""
    from paper_2509_21037_gb300 import host
    prob = synth.cube_heat_3d(2, 5, coef_seed=2) if name == "cubes" else \
        synth.elasticity_cubes((2, 2, 1), 3, 4, seed=3)
    fs = host.factorize_problem(prob.subdomains)
    gpu = feti.FETISolver(prob, fs, device=dev, precond="dirichlet", dirichlet_setup="gpu")
    cpu = feti.FETISolver(prob, fs, device=dev, precond="dirichlet", dirichlet_setup="host")
    for i in range(len(fs)):
        a = gpu.plan.export(gpu.Mdir, i).cpu().numpy()
        b = cpu.plan.export(cpu.Mdir, i).cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), i
    print(f"{name}: Dirichlet set-up GPU {gpu.precond_setup_s:.3f} s vs host {cpu.precond_setup_s:.3f} s")
    if name == "cubes":                       # heat: compatible loads, a solvable interface problem
        loads = feti.compatible_loads(prob, seed=2)
        ra, rb = gpu.solve(loads, tol=1e-10, recover=False), cpu.solve(loads, tol=1e-10, recover=False)
        assert abs(ra.iterations - rb.iterations) <= 1, (ra.iterations, rb.iterations)


def test_graph_chunks_match_the_eager_loop(dev):
    """The loop replayed as CUDA graphs of check_every iterations gives the
    iterations and multipliers of the same steps launched one by one (the
    mixed apply's atomics may order sums differently: 1e-10), and a maxit
    that is no multiple of the chunk length runs the tail eagerly."""
    prob = synth.make_config(2)
    loads = feti.compatible_loads(prob, seed=1)
    g = feti.FETISolver(prob, device=dev, precond="dirichlet")
    e = feti.FETISolver(prob, g.fs, device=dev, precond="dirichlet", graph=False)
    rg = g.solve(loads, tol=1e-10, recover=False)
    re = e.solve(loads, tol=1e-10, recover=False)
    assert g._graph is not None and e._graph is None
    assert abs(rg.iterations - re.iterations) <= 1, (rg.iterations, re.iterations)
    assert np.linalg.norm(rg.lam - re.lam) <= 1e-10 * np.linalg.norm(re.lam)
    print(f"config 2 Dirichlet: graph {rg.solve_ms / rg.iterations:.3f} ms/iteration, "
          f"eager {re.solve_ms / re.iterations:.3f} ms/iteration ({rg.iterations} iterations)")
    short = g.solve(loads, tol=1e-30, maxit=2 * g.check_every + 1, recover=False)
    assert short.iterations == 2 * g.check_every + 1 and len(short.residuals) == short.iterations + 1
