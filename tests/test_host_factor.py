"""The host sparse Cholesky that produces the library's input factor
(paper Sec. 2.2, the numeric stage of K_reg = L L^T).

Pins, each independent of the factor's own code:
  * every stored entry is the correctly rounded result of its column step,
    given the finished entries it depends on: with the stored FP64 entries as
    exact rationals, d = A_jj - sum_k L_jk^2 and s_i = A_ij - sum_k L_ik L_jk
    are formed exactly (fractions.Fraction), and L_jj must equal sqrt(fl(d)),
    L_ij must equal fl(s_i) / L_jj, to one ulp.  Plain FP64 accumulation
    misses this by 6 to ~3e4 ulps on the near-kernel columns of a floating
    subdomain, so a dropped compensation term fails it;
  * backward error ||A - L L^T||_F / ||A||_F near machine precision against
    the dense P K_reg P^T, and agreement with LAPACK's dense Cholesky;
  * structure: CSC lower, diagonal first, rows strictly ascending, fixed dofs
    reduced to an identity column and row;
  * a matrix with a negative eigenvalue is rejected;
  * the two stages apart (scf_analyze once, scf_numeric per set of values)
    give scf_factorize's factor bit for bit, and K -> 4 K gives L -> 2 L
    exactly, also with several threads sharing one analysis.
The cases span the supernode shapes the factor takes: single columns, panels
whose width is not a multiple of four, and one dense panel of width 37.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from paper_2509_21037_gb300 import host


def _kreg(K, fixed):
    A = sp.csr_matrix(K).toarray()
    for d in fixed:
        A[d, :] = 0.0
        A[:, d] = 0.0
        A[d, d] = 1.0
    return A


def _random_spd(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, data_rvs=lambda k: rng.uniform(-1, 1, k)).toarray()
    M = np.tril(M, -1)
    M = M + M.T
    M += np.diag(np.abs(M).sum(axis=1) + 1.0)
    return sp.csr_matrix(M)


def _chain(n):
    main = np.full(n, 2.0)
    main[-1] = 1.0
    return sp.diags([main, -np.ones(n - 1), -np.ones(n - 1)], [0, 1, -1], format="csr")


def _cases():
    c1 = synth.make_config(1).subdomains[0]
    yield "heat2d_k16", c1.K, c1.fixed, None
    sd = synth.cube_heat_3d(1, 5).subdomains[0]
    yield "heat3d_k5", sd.K, sd.fixed, None
    el = synth.elasticity_cubes((1, 1, 1), 3, 3, seed=1).subdomains[0]
    yield "elast_k3", el.K, el.fixed, None
    yield "random_spd", _random_spd(90, 0.05, 3), np.array([], np.int64), None
    D = _random_spd(37, 1.0, 5)
    yield "dense37", D, np.array([], np.int64), np.arange(37)
    yield "chain50", _chain(50), np.array([0]), np.arange(50)


CASES = list(_cases())


def _factor(K, fixed, perm):
    return host.factorize(K, fixed, perm=perm, postorder=perm is None)


def _supernode_widths(f):
    cnt = np.diff(f.colptr)
    parent = np.array([f.rowind[f.colptr[j] + 1] if cnt[j] > 1 else -1 for j in range(f.n)])
    starts = [0] + [j for j in range(1, f.n) if not (parent[j - 1] == j and cnt[j - 1] == cnt[j] + 1)]
    return np.diff(starts + [f.n])


def test_cases_span_the_supernode_shapes():
    widths = np.concatenate([_supernode_widths(_factor(K, fx, p)) for _, K, fx, p in CASES])
    assert (widths == 1).any()
    assert ((widths > 4) & (widths % 4 != 0)).any()
    assert widths.max() >= 37


@pytest.mark.parametrize("name,K,fixed,perm", CASES, ids=[c[0] for c in CASES])
def test_structure_and_backward_error(name, K, fixed, perm):
    f = _factor(K, fixed, perm)
    n = f.n
    assert sorted(f.perm.tolist()) == list(range(n))
    for j in range(n):
        rows = f.rowind[f.colptr[j]:f.colptr[j + 1]]
        assert rows[0] == j and np.all(np.diff(rows) > 0)
    A = _kreg(K, fixed)[np.ix_(f.perm, f.perm)]
    L = sp.csc_matrix((f.values, f.rowind, f.colptr), shape=(n, n)).toarray()
    assert np.linalg.norm(A - L @ L.T) <= 1e-15 * math.sqrt(n) * np.linalg.norm(A)
    Ld = np.linalg.cholesky(A)
    assert np.linalg.norm(L - Ld) <= 1e-12 * np.linalg.norm(Ld)
    inv = np.empty(n, np.int64)
    inv[f.perm] = np.arange(n)
    for d in fixed:
        j = inv[d]
        assert f.colptr[j + 1] - f.colptr[j] == 1 and f.values[f.colptr[j]] == 1.0
        assert not np.any(L[j, :j])


@pytest.mark.parametrize("name,K,fixed,perm", CASES, ids=[c[0] for c in CASES])
def test_every_entry_is_its_correctly_rounded_column_step(name, K, fixed, perm):
    f = _factor(K, fixed, perm)
    n, cp, ri, v = f.n, f.colptr, f.rowind, f.values
    A = _kreg(K, fixed)[np.ix_(f.perm, f.perm)]
    col = [dict(zip(ri[cp[j]:cp[j + 1]].tolist(), v[cp[j]:cp[j + 1]].tolist())) for j in range(n)]
    left = [[] for _ in range(n)]                 # columns k < j with L_jk != 0
    for k in range(n):
        for i in ri[cp[k] + 1:cp[k + 1]]:
            left[i].append(k)
    worst = 0.0
    for j in range(n):
        ljj = col[j][j]
        for i in ri[cp[j]:cp[j + 1]].tolist():
            s = Fraction(A[i, j])
            for k in left[j]:
                lik = col[k].get(i)
                if lik is not None:
                    s -= Fraction(lik) * Fraction(col[k][j])
            ref = math.sqrt(float(s)) if i == j else float(s) / ljj
            if ref != 0.0:
                worst = max(worst, abs(col[j][i] - ref) / np.spacing(abs(ref)))
            else:
                assert col[j][i] == 0.0
    assert worst <= 1.0, f"{name}: an entry is {worst} ulps from its correctly rounded column step"


def test_indefinite_matrix_is_rejected():
    K = _chain(20).tolil()
    K[10, 10] = -1.0
    with pytest.raises(RuntimeError):
        host.factorize(sp.csr_matrix(K), [], perm=np.arange(20), postorder=False)


@pytest.mark.parametrize("name,K,fixed,perm", CASES, ids=[c[0] for c in CASES])
def test_numeric_stage_alone_reproduces_factorize(name, K, fixed, perm):
    """scf_analyze once + scf_numeric gives scf_factorize's factor bit for bit;
    K -> 4 K gives L -> 2 L exactly on the free columns (every product, sum,
    square root and quotient of the numeric stage scales exactly by powers of
    two), while the fixed dofs keep their unit columns."""
    sym = host.SymbolicFactor(K, fixed, perm=perm, postorder=perm is None)
    f = _factor(K, fixed, perm)
    g = sym.numeric(K)
    assert np.array_equal(g.perm, f.perm) and np.array_equal(g.colptr, f.colptr)
    assert np.array_equal(g.rowind, f.rowind) and np.array_equal(g.values, f.values)
    g4 = sym.numeric(sp.csr_matrix(K) * 4.0)
    inv = np.empty(f.n, np.int64)
    inv[f.perm] = np.arange(f.n)
    fixed_cols = set(inv[np.asarray(fixed, np.int64)].tolist())
    col_of = np.repeat(np.arange(f.n), np.diff(f.colptr))
    free = np.array([c not in fixed_cols for c in col_of])
    assert np.array_equal(g4.values[free], 2.0 * f.values[free])
    assert np.array_equal(g4.values[~free], f.values[~free])


def test_numeric_stage_threads_share_one_analysis():
    """scf_numeric only reads the handle: concurrent calls with different
    values give each its own factor."""
    from concurrent.futures import ThreadPoolExecutor
    sd = synth.cube_heat_3d(1, 6).subdomains[0]
    sym = host.SymbolicFactor(sd.K, sd.fixed)
    scales = [1.0, 4.0, 0.25, 16.0, 1.0, 4.0]
    with ThreadPoolExecutor(4) as ex:
        outs = list(ex.map(lambda c: sym.numeric(sd.K * c).values, scales))
    ref = sym.numeric(sd.K).values
    free = ref != 1.0
    for c, v in zip(scales, outs):
        assert np.array_equal(v[free], math.sqrt(c) * ref[free])


def test_symbolic_and_numeric_reject_bad_input():
    K = _chain(12)
    sym = host.SymbolicFactor(K, [0], perm=np.arange(12), postorder=False)
    with pytest.raises(ValueError):
        sym.numeric(K + sp.eye(12, k=3))                   # another pattern
    with pytest.raises(RuntimeError):
        sym.numeric(-K)                                    # not SPD
    bad = sp.csc_matrix(K)
    bad.indices = bad.indices.copy()
    bad.indices[5] = 40                                    # row index out of range
    with pytest.raises(RuntimeError):
        host.SymbolicFactor(bad, [0], perm=np.arange(12), postorder=False)


def test_solve_LLt_against_scipy_triangular_solves():
    """host.solve_LLt (scf_solve) against scipy's sparse triangular solves
    on the same factor; bad patterns are refused."""
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(3)
    for name, K, fixed, perm in CASES[:3]:
        f = _factor(K, fixed, perm)
        L = sp.csr_matrix(sp.csc_matrix((f.values, f.rowind, f.colptr), shape=(f.n, f.n)))
        b = rng.standard_normal(f.n)
        ref = spla.spsolve_triangular(L.T.tocsr(), spla.spsolve_triangular(L, b, lower=True), lower=False)
        x = host.solve_LLt(f, b)
        assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref), name
    bad = host.HostFactor(f.n, f.colptr, f.rowind.copy(), f.values, f.perm)
    bad.rowind[f.colptr[4]] += 1                           # column 4 no longer starts with its diagonal
    with pytest.raises(RuntimeError):
        host.solve_LLt(bad, b)
