"""CPU pins of the FETI-1 formulation that the PCPG solver (feti.py) runs on
the library's F: kernel bases, the fixed-dof correction of the generalised
inverse, and a projected CG on the oracle's F that recovers a continuous,
equilibrated primal solution."""
import numpy as np
import scipy.sparse as sp

import oracle
import synth
from paper_2509_21037_gb300 import feti, host


def test_kernel_bases_span_ker_K():
    for prob, r in ((synth.cube_heat_3d(2, 4), 1), (synth.elasticity_cubes((2, 1, 1), 3, 3, seed=0), 6)):
        for sd in prob.subdomains:
            R = feti.kernel_basis(sd)
            K = sd.K.toarray()
            assert np.abs(K @ R).max() <= 1e-12 * np.abs(K).max()
            assert np.linalg.matrix_rank(R) == r
            # the fixed set is minimal: K restricted to the free dofs is nonsingular
            free = np.setdiff1d(np.arange(K.shape[0]), sd.fixed)
            assert np.linalg.matrix_rank(K[np.ix_(free, free)]) == K.shape[0] - len(sd.fixed) == K.shape[0] - r


def _kplus_dense(sd):
    """The generalised inverse zero on the fixed dofs (K K^+ K = K)."""
    K = sd.K.toarray()
    n = K.shape[0]
    free = np.setdiff1d(np.arange(n), sd.fixed)
    Kp = np.zeros((n, n))
    Kp[np.ix_(free, free)] = np.linalg.inv(K[np.ix_(free, free)])
    return K, Kp


def _dual_problem(prob, loads):
    """F (from the oracle, corrected), G, d, e of the interface problem."""
    nd = prob.n_dual
    Fo = oracle.dual_operators(prob.subdomains)
    F = np.zeros((nd, nd))
    G, d, e = [], np.zeros(nd), []
    for sd, Fi, f in zip(prob.subdomains, Fo, loads):
        lm = np.asarray(sd.lambda_map)
        Bt = sd.Bt.toarray()
        K, Kp = _kplus_dense(sd)
        assert np.allclose(K @ Kp @ K, K, atol=1e-9 * np.abs(K).max())
        # the library's operator is built from K_reg^{-1} = K^+ + E_f
        Ef = np.zeros_like(K)
        Ef[sd.fixed, sd.fixed] = 1.0
        assert np.allclose(Fi - Bt.T @ Ef @ Bt, Bt.T @ Kp @ Bt, rtol=0, atol=1e-10 * np.abs(Fi).max())
        F[np.ix_(lm, lm)] += Fi - Bt.T @ Ef @ Bt
        R = feti.kernel_basis(sd)
        g = np.zeros((nd, R.shape[1]))
        g[lm] = Bt.T @ R
        G.append(g)
        d[lm] += Bt.T @ (Kp @ f)
        e.append(R.T @ f)
    return F, np.hstack(G), d, np.concatenate(e)


def test_projected_cg_on_oracle_operator_solves_the_decomposed_problem():
    prob = synth.cube_heat_3d(2, 4, coef_seed=3)
    loads = feti.compatible_loads(prob, seed=5)
    F, G, d, e = _dual_problem(prob, loads)
    GtGp = np.linalg.pinv(G.T @ G, rcond=1e-12, hermitian=True)
    P = lambda x: x - G @ (GtGp @ (G.T @ x))
    lam = G @ (GtGp @ e)
    assert np.allclose(G.T @ lam, e)
    r = d - F @ lam
    w = P(r)
    p, zw_old = None, None
    for _ in range(500):
        z = w
        zw = z @ w
        p = z if p is None else z + zw / zw_old * p
        q = F @ p
        eta = zw / (p @ q)
        lam, r = lam + eta * p, r - eta * q
        w, zw_old = P(r), zw
        if np.linalg.norm(w) < 1e-12 * np.linalg.norm(d):
            break
    alpha = GtGp @ (G.T @ (F @ lam - d))
    us, k = [], 0
    jump = np.zeros(prob.n_dual)
    for sd, f in zip(prob.subdomains, loads):
        K, Kp = _kplus_dense(sd)
        R = feti.kernel_basis(sd)
        lm = np.asarray(sd.lambda_map)
        Bt = sd.Bt.toarray()
        u = Kp @ (f - Bt @ lam[lm]) + R @ alpha[k:k + R.shape[1]]
        k += R.shape[1]
        assert np.linalg.norm(K @ u - f + Bt @ lam[lm]) <= 1e-9 * np.linalg.norm(f)   # equilibrium
        jump[lm] += Bt.T @ u
        us.append(u)
    assert np.linalg.norm(jump) <= 1e-9 * max(np.linalg.norm(u) for u in us)        # continuity


def test_schur_on_glued_dofs():
    """S_i (feti.schur_on_glued) against its definition through the harmonic
    extension, solved independently with a sparse LU: S u_b = K_bb u_b +
    K_bi u_i with K_ii u_i = -K_ib u_b; S annihilates the rigid-body modes
    restricted to the glued dofs and is positive semidefinite."""
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(2)
    for prob in (synth.cube_heat_3d(2, 4, coef_seed=1), synth.elasticity_cubes((2, 1, 1), 3, 3, seed=0)):
        for sd in prob.subdomains[:2]:
            S = feti.schur_on_glued(sd)
            b = feti.glued_dofs(sd)
            K = sp.csr_matrix(sd.K)
            i = np.setdiff1d(np.arange(K.shape[0]), b)
            lu = spla.splu(sp.csc_matrix(K[i][:, i]))
            for _ in range(3):
                ub = rng.standard_normal(len(b))
                ui = lu.solve(-(K[i][:, b] @ ub))
                ref = K[b][:, b] @ ub + K[b][:, i] @ ui
                assert np.linalg.norm(S @ ub - ref) <= 1e-10 * np.linalg.norm(ref)
            R = feti.kernel_basis(sd)[b]
            assert np.abs(S @ R).max() <= 1e-9 * np.abs(S).max() * np.abs(R).max()
            assert np.linalg.eigvalsh(S).min() >= -1e-10 * np.abs(S).max()


def _pcpg(F, G, d, e, precond=None, tol=1e-10, maxit=500):
    GtGp = np.linalg.pinv(G.T @ G, rcond=1e-12, hermitian=True)
    P = lambda x: x - G @ (GtGp @ (G.T @ x))
    lam = G @ (GtGp @ e)
    r = d - F @ lam
    w = P(r)
    w0 = np.linalg.norm(w)
    p, zw_old = None, None
    for it in range(1, maxit + 1):
        z = w if precond is None else P(precond @ w)
        zw = z @ w
        p = z if p is None else z + zw / zw_old * p
        q = F @ p
        eta = zw / (p @ q)
        lam, r = lam + eta * p, r - eta * q
        w, zw_old = P(r), zw
        if np.linalg.norm(w) < tol * w0:
            return lam, it
    raise AssertionError("PCPG did not converge")


def _bbt(prob):
    nd = prob.n_dual
    BB = np.zeros((nd, nd))
    for sd in prob.subdomains:
        lm = np.asarray(sd.lambda_map)
        Bt = sd.Bt.toarray()
        BB[np.ix_(lm, lm)] += Bt.T @ Bt
    return BB


def test_bbt_inverse_is_the_pseudo_inverse():
    """feti.bbt_inverse against numpy's dense pseudo-inverse of B B^T: heat
    (non-redundant gluing, B B^T invertible) and an elasticity lattice whose
    multipliers close loops (B B^T singular)."""
    for prob in (synth.cube_heat_3d(3, 3), synth.elasticity_cubes((2, 2, 1), 3, 3, seed=0)):
        BB = _bbt(prob)
        W = feti.bbt_inverse(prob.subdomains, prob.n_dual).toarray()
        assert np.abs(W - np.linalg.pinv(BB, hermitian=True)).max() <= 1e-13
    assert np.linalg.matrix_rank(_bbt(synth.elasticity_cubes((2, 2, 1), 3, 3, seed=0))) < 192


def test_scaled_preconditioners_cut_iterations():
    """PCPG on the oracle's operator with the Dirichlet preconditioner
    W (sum_i B_i S_i B_i^T) W (blocks from feti.dirichlet_block, scattered by
    the lambda maps) and the lumped W (sum_i B_i K_i B_i^T) W, W = (B B^T)^+
    computed here densely: both converge to the multipliers of the
    unpreconditioned solve, Dirichlet in the fewest iterations; without W the
    same sums take more iterations than no preconditioner (the non-redundant
    gluing weights edge and corner multipliers wrongly)."""
    prob = synth.cube_heat_3d(3, 4, coef_seed=3)
    loads = feti.compatible_loads(prob, seed=5)
    F, G, d, e = _dual_problem(prob, loads)
    nd = prob.n_dual
    MD = np.zeros((nd, nd))
    ML = np.zeros((nd, nd))
    for sd in prob.subdomains:
        lm = np.asarray(sd.lambda_map)
        Bt = sd.Bt.toarray()
        MD[np.ix_(lm, lm)] += feti.dirichlet_block(sd)
        ML[np.ix_(lm, lm)] += Bt.T @ sd.K.toarray() @ Bt
    W = np.linalg.pinv(_bbt(prob), hermitian=True)
    lam0, n0 = _pcpg(F, G, d, e)
    lamL, nL = _pcpg(F, G, d, e, W @ ML @ W)
    lamD, nD = _pcpg(F, G, d, e, W @ MD @ W)
    for lam in (lamL, lamD):
        assert np.linalg.norm(lam - lam0) <= 1e-7 * np.linalg.norm(lam0)
    assert nD < nL < n0 // 3, (nD, nL, n0)
    assert _pcpg(F, G, d, e, ML)[1] > n0 and _pcpg(F, G, d, e, MD)[1] > n0


class _DenseFETI(feti.FETISolver):
    """feti.FETISolver's host-side logic on the CPU: the library's plan is
    replaced by dense products with the oracle's operator (F = sum_i B_i
    K_reg^-1 B_i^T scattered by the lambda maps; pack assembles the blocks
    the same way), everything else -- projector, fixed-dof correction,
    scalings, preconditioners, PCPG, recovery -- is the solver's own code."""

    def _make_operator(self, plan_kwargs):
        import torch
        nd = self.nd
        Fd = np.zeros((nd, nd))
        for sd, Fi in zip(self.subs, oracle.dual_operators(self.subs)):
            lm = np.asarray(sd.lambda_map)
            Fd[np.ix_(lm, lm)] += Fi
        subs = self.subs

        class _Plan:
            def apply(self, F, x, q, stream=None):
                q.copy_(F @ x)

            def pack(self, blocks, device):
                M = np.zeros((nd, nd))
                for sd, Bk in zip(subs, blocks):
                    lm = np.asarray(sd.lambda_map)
                    M[np.ix_(lm, lm)] += Bk
                return torch.from_numpy(M)

            def add_symmetric(self, F, i, rows, cols, vals):
                lm = np.asarray(subs[i].lambda_map)
                for r, c, v in zip(rows, cols, vals):
                    F[lm[r], lm[c]] += v
                    if r != c:
                        F[lm[c], lm[r]] += v

        return _Plan(), torch.from_numpy(Fd)


def test_feti_solver_logic_on_the_cpu():
    """The solver with each preconditioner reaches the multipliers of a plain
    projected CG on the oracle's operator, recovers a continuous and
    equilibrated primal solution, orders the iteration counts Dirichlet <
    lumped < none, and a solve without recovery (the bench's warm-up) gives
    the same iterations and multipliers."""
    import math
    pytest = __import__("pytest")
    pytest.importorskip("torch")
    prob = synth.cube_heat_3d(2, 4, coef_seed=3)
    loads = feti.compatible_loads(prob, seed=5)
    fs = host.factorize_problem(prob.subdomains)
    F, G, d, e = _dual_problem(prob, loads)
    lam_ref, _ = _pcpg(F, G, d, e, tol=1e-12)
    its = {}
    for pc in ("none", "lumped", "dirichlet"):
        s = _DenseFETI(prob, fs, device="cpu", precond=pc)
        r0 = s.solve(loads, tol=1e-10, recover=False)
        assert math.isnan(r0.continuity) and r0.u == [] and r0.solve_ms >= 0 and r0.apply_ms >= 0
        r = s.solve(loads, tol=1e-10)
        assert r.iterations == r0.iterations and np.array_equal(r.lam, r0.lam)
        assert np.linalg.norm(r.lam - lam_ref) <= 1e-7 * np.linalg.norm(lam_ref)
        assert r.continuity <= 1e-8 and r.equilibrium <= 1e-8
        its[pc] = r.iterations
    assert its["dirichlet"] < its["lumped"] < its["none"], its


def test_dirichlet_blocks_through_the_library_plan():
    """The Dirichlet preconditioner's blocks as this library's problem
    (interior factor + general right-hand side C_i = K_ib B_b^T, include/sc.h
    Bt_val): the plan replayed on the CPU gives C_i^T K_ii^{-1} C_i, and
    K_bb's gather minus it equals the dense host Schur complement
    (schur_on_glued / dirichlet_block) block by block."""
    import plan_emulator as pe
    from paper_2509_21037_gb300 import sc
    for prob in (synth.cube_heat_3d(parts=2, k=4), synth.elasticity_cubes((2, 2, 1), 2, 3, seed=1)):
        facs, kbb = feti.dirichlet_problem(prob.subdomains, threads=1)
        plan = sc.Plan(facs, prob.n_dual)
        T = pe.export_plan(plan)
        pe.check_bounds(T, plan.sizes, plan.stats)
        Fc = pe.emulate_assembly(T, plan.sizes, plan.stats, sc.concat_L_values(facs))
        for i, sd in enumerate(prob.subdomains):
            r, c, v = kbb[i]
            assert np.all(r >= c)
            Kb = np.zeros((plan.m[i], plan.m[i]))
            np.add.at(Kb, (r, c), v)
            Kb = Kb + np.tril(Kb, -1).T
            M = Kb - pe.export_dense(T, Fc, i)
            ref = feti.dirichlet_block(sd)
            assert np.linalg.norm(M - ref) <= 1e-12 * np.linalg.norm(ref), i
