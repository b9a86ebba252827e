"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

* closed form: 1D chain with node 0 fixed, K^{-1}_{ij} = h min(i, j);
* brute force: numpy.linalg.inv(K_reg) gathered by B on tiny grids;
* independent solve: conjugate gradients on sparse K_reg for F lambda;
* invariants: symmetry, PSD, coefficient scaling, fixed-dof rows,
  duplicate-dof columns;
* planted mistakes: each plausible slip in the oracle makes a pin fail.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth


def _brute(sd):
    A = np.asarray(sd.K.todense(), float)
    f = np.asarray(sd.fixed)
    A[f, :] = 0
    A[:, f] = 0
    A[f, f] = 1
    Bt = sd.Bt.toarray()
    return Bt.T @ np.linalg.inv(A) @ Bt


def _random_bt_subdomain(sd, m, seed, multi=False):
    """Same K, random B^T: signed unit columns, duplicates allowed, optionally
    a few columns with several nonzeros (general gluing)."""
    rng = np.random.default_rng(seed)
    n = sd.n
    rows, cols, vals = [], [], []
    for j in range(m):
        k = rng.integers(1, 4) if (multi and j % 5 == 0) else 1
        for r in rng.choice(n, size=k, replace=False):
            rows.append(r)
            cols.append(j)
            vals.append(rng.choice([-1.0, 1.0]))
    Bt = sp.csc_matrix((vals, (rows, cols)), shape=(n, m))
    return synth.Subdomain(K=sd.K, fixed=sd.fixed, Bt=Bt, lambda_map=np.arange(m),
                           grid=sd.grid, ndpn=sd.ndpn, key=None)


# ---------------------------------------------------------------- closed form

@pytest.mark.parametrize("nel", [1, 7, 40])
def test_chain_closed_form(nel):
    rng = np.random.default_rng(nel)
    sel = rng.integers(0, nel + 1, size=12)
    sel[0] = 0                                    # the fixed node is selected too
    signs = rng.choice([-1.0, 1.0], size=12)
    sd = synth.chain_1d(nel, sel, signs)
    F = oracle.dual_operator(sd)
    h = 1.0 / nel
    ref = np.empty((12, 12))
    for a in range(12):
        for b in range(12):
            ia, ib = sel[a], sel[b]
            if ia == 0 or ib == 0:                 # fixed dof: K_reg^{-1} e_0 = e_0
                g = 1.0 if ia == ib else 0.0
            else:
                g = h * min(ia, ib)
            ref[a, b] = signs[a] * signs[b] * g
    assert np.max(np.abs(F - ref)) <= 1e-13 * max(1.0, np.abs(ref).max())


def test_refinement_reaches_closed_form_on_ill_conditioned_chain():
    """A long chain (kappa(K_reg) ~ 1e7): the plain FP64 solve misses the
    closed form h*min(i,j) by ~1e-10; one refinement step with the exact
    residual recovers it to ~1e-15 relative."""
    nel = 3000
    sel = np.array([1, 17, 700, 1500, 2999, 3000])
    sd = synth.chain_1d(nel, sel)
    h = 1.0 / nel
    ref = h * np.minimum.outer(sel, sel).astype(float)
    e0 = oracle.relative_frobenius(oracle.dual_operator(sd, refine=0), ref)
    e1 = oracle.relative_frobenius(oracle.dual_operator(sd, refine=1), ref)
    assert e1 <= 1e-14 and e1 < e0


def test_residual_is_exact_against_rationals():
    from fractions import Fraction
    rng = np.random.default_rng(5)
    A = sp.random(12, 12, density=0.4, random_state=3, format="csr") + sp.eye(12)
    A.data = rng.standard_normal(A.nnz) * 10.0 ** rng.integers(-8, 8, A.nnz)
    X = rng.standard_normal((12, 3)) * 10.0 ** rng.integers(-8, 8, (12, 3))
    R0 = rng.standard_normal((12, 3))
    got = oracle.residual(A, X, R0)
    Ad = A.toarray()
    for i in range(12):
        for c in range(3):
            exact = Fraction(R0[i, c]) - sum(Fraction(Ad[i, k]) * Fraction(X[k, c]) for k in range(12))
            assert abs(got[i, c] - float(exact)) <= np.spacing(abs(float(exact)))   # within one ulp of exact


# ---------------------------------------------------------------- brute force

def _tiny_cases():
    out = []
    for k in (2, 3, 4):
        out.append(("q1_%d" % k, synth.single_heat_2d(k).subdomains[0]))
    out.append(("config1", synth.single_heat_2d(16).subdomains[0]))
    p = synth.cube_heat_3d(parts=2, k=2)
    out += [("hex_%d" % i, s) for i, s in enumerate(p.subdomains[:3])]
    p = synth.elasticity_cubes((2, 1, 1), 1, 2, seed=3)
    out += [("elast_%d" % i, s) for i, s in enumerate(p.subdomains)]
    return out


@pytest.mark.parametrize("name,sd", _tiny_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_brute_force_inverse(name, sd):
    F = oracle.dual_operator(sd)
    ref = _brute(sd)
    assert oracle.relative_frobenius(F, ref) < 1e-13


@pytest.mark.parametrize("multi", [False, True])
def test_brute_force_general_bt(multi):
    base = synth.elasticity_cubes((1, 1, 1), 2, 2, seed=1).subdomains[0]
    sd = _random_bt_subdomain(base, 30, seed=11, multi=multi)
    assert oracle.relative_frobenius(oracle.dual_operator(sd), _brute(sd)) < 1e-12


def test_cholesky_against_definition():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((150, 150))
    A = M @ M.T + 150 * np.eye(150)
    G = oracle.cholesky(A, block=32)
    assert np.allclose(np.triu(G, 1), 0)
    assert np.abs(G @ G.T - A).max() < 1e-11 * np.abs(A).max()
    with pytest.raises(oracle.NotSPDError):
        oracle.cholesky(-A)


# ---------------------------------------------------------------- independent solve

def _cg_apply(sd, lam):
    """B K_reg^{-1} B^T lambda by conjugate gradients on sparse K_reg (no factorisation)."""
    K = sp.lil_matrix(sd.K, dtype=float)
    for f in sd.fixed:
        K[f, :] = 0
        K[:, f] = 0
        K[f, f] = 1
    K = K.tocsr()
    rhs = sd.Bt @ lam
    x, info = spla.cg(K, rhs, rtol=1e-15, atol=0.0, maxiter=20000)
    assert info == 0 or np.linalg.norm(K @ x - rhs) < 1e-12 * np.linalg.norm(rhs)
    return sd.Bt.T @ x


@pytest.mark.parametrize("which", ["config1", "heat3d", "elast"])
def test_apply_matches_cg(which):
    if which == "config1":
        sd = synth.make_config(1).subdomains[0]
    elif which == "heat3d":
        sd = synth.cube_heat_3d(parts=2, k=5).subdomains[3]
    else:
        sd = synth.elasticity_cubes((2, 1, 1), 3, 3, seed=2).subdomains[0]
    F = oracle.dual_operator(sd)
    lam = np.random.default_rng(5).standard_normal(sd.m)
    ref = _cg_apply(sd, lam)
    assert np.linalg.norm(F @ lam - ref) <= 1e-10 * np.linalg.norm(ref)


# ---------------------------------------------------------------- invariants

def test_symmetry_and_psd_config1():
    F = oracle.dual_operator(synth.make_config(1).subdomains[0])
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()
    ev = np.linalg.eigvalsh(0.5 * (F + F.T))
    assert ev.min() >= -1e-12 * ev.max()


def test_duplicate_dofs_and_fixed_rows():
    p = synth.cube_heat_3d(parts=2, k=3)
    for sd in p.subdomains:
        F = oracle.dual_operator(sd)
        dof = sd.Bt.indices
        sgn = sd.Bt.data
        for a in range(sd.m):
            same = np.nonzero(dof == dof[a])[0]
            for b in same:                      # columns on the same dof: equal up to sign
                assert np.allclose(F[:, a] * sgn[a], F[:, b] * sgn[b], rtol=0, atol=1e-13)
            if dof[a] in sd.fixed:              # fixed dof: row is +-1 on its own dof, else 0
                expect = np.where(dof == dof[a], sgn * sgn[a], 0.0)
                assert np.allclose(F[a], expect, atol=1e-14)


def test_coefficient_scaling():
    """K -> c K leaves the fixed-dof block alone and scales the rest of F by 1/c."""
    unit = synth.cube_heat_3d(parts=2, k=3)
    scaled = synth.cube_heat_3d(parts=2, k=3, coef_seed=9)
    memo = oracle._Memo()
    for su, ss in zip(unit.subdomains, scaled.subdomains):
        c = ss.K[0, 0] / su.K[0, 0]
        assert not np.isclose(c, 1.0)
        Fu = oracle.dual_operator(su, memo)
        Fs = oracle.dual_operator(ss, memo)
        fixed = np.isin(su.Bt.indices, su.fixed)
        free = ~fixed
        assert np.allclose(Fs[np.ix_(free, free)], Fu[np.ix_(free, free)] / c, rtol=1e-12, atol=0)
        assert np.allclose(Fs[np.ix_(fixed, fixed)], Fu[np.ix_(fixed, fixed)], atol=1e-15)


def test_sampled_columns_against_brute_force():
    sd = synth.elasticity_cubes((2, 1, 1), 2, 3, seed=4).subdomains[1]
    cols = [0, 5, sd.m - 1]
    assert oracle.relative_frobenius(oracle.dual_operator_columns(sd, cols), _brute(sd)[:, cols]) < 1e-12


def test_apply_dual_sums_subdomains():
    p = synth.cube_heat_3d(parts=2, k=2)
    Fs = oracle.dual_operators(p.subdomains)
    lam = np.random.default_rng(1).standard_normal(p.n_dual)
    q = oracle.apply_dual(Fs, [s.lambda_map for s in p.subdomains], lam, p.n_dual)
    ref = np.zeros(p.n_dual)
    for s, F in zip(p.subdomains, Fs):
        Bfull = np.zeros((s.m, p.n_dual))
        Bfull[np.arange(s.m), s.lambda_map] = 1.0
        ref += Bfull.T @ F @ Bfull @ lam
    assert np.allclose(q, ref, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- planted mistakes

def _pins_pass():
    try:
        test_chain_closed_form(7)
        for name, sd in _tiny_cases()[:4]:
            test_brute_force_inverse(name, sd)
        return True
    except (AssertionError, oracle.NotSPDError, ValueError, FloatingPointError):
        return False


def _bad_regularize(K, f):
    A = _ORIG["regularize"](K, f)
    A[np.asarray(f), np.asarray(f)] = 2.0          # wrong diagonal on fixed dofs
    return A


def _bad_backward(G, Z, block=64):
    return oracle.forward_substitution(G, Z, block)  # G^{-1} where G^{-T} belongs


def _bad_cholesky(A, block=64):
    A = np.array(A, float)                          # trailing update dropped
    n = A.shape[0]
    for k0 in range(0, n, block):
        k1 = min(k0 + block, n)
        Gkk = oracle._cholesky_unblocked(A[k0:k1, k0:k1])
        A[k0:k1, k0:k1] = Gkk
        if k1 < n:
            A[k1:, k0:k1] = oracle._lower_solve_small(Gkk, A[k1:, k0:k1].T).T
    return np.tril(A)


def _unsigned_dual_operator(sd, memo=None):
    sd2 = synth.Subdomain(K=sd.K, fixed=sd.fixed, Bt=abs(sd.Bt), lambda_map=sd.lambda_map,
                          grid=sd.grid, ndpn=sd.ndpn, key=None)
    return _ORIG["dual_operator"](sd2, memo)     # signs of B dropped


_ORIG = {"regularize": oracle.regularize, "dual_operator": oracle.dual_operator}


@pytest.mark.parametrize("name,bad", [("regularize", _bad_regularize),
                                      ("backward_substitution", _bad_backward),
                                      ("cholesky", _bad_cholesky),
                                      ("dual_operator", _unsigned_dual_operator)])
def test_pins_catch_planted_mistakes(monkeypatch, name, bad):
    assert _pins_pass()
    monkeypatch.setattr(oracle, name, bad)
    assert not _pins_pass()


def test_config1_anchor_golden():
    """The oracle's config-1 F against the stored anchor (written by
    tests/golden/make_config1_anchor.py from the oracle) and against an
    independent dense computation's printed digits."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config1_anchor.txt")
    stored = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        stored[k] = float(v)
    F = oracle.dual_operator(synth.make_config(1).subdomains[0], refine=1)
    ev = np.linalg.eigvalsh(0.5 * (F + F.T))
    got = {"frobenius": np.linalg.norm(F), "trace": np.trace(F), "lambda_min": ev[0], "lambda_max": ev[-1],
           "m": F.shape[0]}
    for k, v in stored.items():
        assert abs(got[k] - v) <= 1e-12 * max(1.0, abs(v)), k
    # independent dense computation (numpy inverse of K_reg gathered by B), 4-5 printed digits
    assert abs(got["frobenius"] - 174.9015) < 5e-5
    assert abs(got["trace"] - 266.3118) < 5e-5
    assert abs(got["lambda_min"] - 0.5774) < 5e-5
    assert abs(got["lambda_max"] - 173.8) < 5e-2


def test_residual_c_and_numpy_forms_bit_identical():
    """oracle/residual.c runs the loops of residual_numpy; on inputs spanning
    16 decades the two agree bit for bit (and the numpy form is the one the
    rational-arithmetic pin above also checks through this equality)."""
    if not oracle.build_c():
        pytest.skip("no C compiler")
    rng = np.random.default_rng(9)
    A = sp.random(400, 400, density=0.03, random_state=4, format="csr") + sp.eye(400)
    A.data = rng.standard_normal(A.nnz) * 10.0 ** rng.integers(-8, 8, A.nnz)
    X = rng.standard_normal((400, 7)) * 10.0 ** rng.integers(-8, 8, (400, 7))
    R0 = rng.standard_normal((400, 7))
    assert np.array_equal(oracle.residual(A, X, R0), oracle.residual_numpy(A, X, R0))
    assert np.array_equal(oracle.residual(A, X[:, 0], R0[:, 0]), oracle.residual_numpy(A, X[:, :1], R0[:, :1])[:, 0])
