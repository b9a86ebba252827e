"""CPU pins of the FETI-1 formulation that the PCPG solver (feti.py) runs on
the library's F: kernel bases, the fixed-dof correction of the generalised
inverse, and a projected CG on the oracle's F that recovers a continuous,
equilibrated primal solution."""
import numpy as np
import scipy.sparse as sp

import oracle
import synth
from paper_2509_21037_gb300 import feti


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
