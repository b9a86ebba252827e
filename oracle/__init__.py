"""FP64 CPU oracle for the explicit FETI dual operator -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run this package.  The
library (``paper_2509_21037_gb300``) never imports it and shares no code with
it: the oracle never sees the sparse factor ``L``, the fill-reducing
permutation, the column pivots or any tile/supernode structure.

What it computes is the plain definition of the local dual operator
(paper Sec. 2.1, Eq. "localdualoperator" and Eq. "localdualoperatorwithU"):

    F_i = B_i K_i^+ B_i^T,      K_i^+ = K_{i,reg}^{-1},

in FP64, by

  1. ``regularize``   -- K_reg from K and the fixed dofs (fixing-node reading:
                         fixed rows and columns replaced by the identity);
  2. ``cholesky``     -- dense blocked Cholesky K_reg = G G^T written out here
                         (the only library primitive used is the matrix product);
  3. ``solve_spd``    -- forward then backward substitution with G on the
                         distinct dofs touched by B^T;
  4. ``dual_operator``-- F = B X, returned as a full symmetric m x m matrix;
                         optionally after iterative refinement of X with an
                         error-free residual (``refine`` steps), because for
                         floating subdomains fixed at few dofs kappa(K_reg)
                         reaches 1e6 and a plain FP64 solve is then only good
                         to ~1e-12;
  5. ``apply_dual``   -- q = sum_i scatter_i(F_i gather_i(lambda))
                         (paper Eq. "dualop_apply_expl" summed over subdomains).

Parity status: pinned.  The tests pin it to the 1D-chain closed form
K^{-1}_{ij} = h min(i, j), to brute-force ``numpy.linalg.inv`` on tiny grids, to
an independent conjugate-gradient solve of K_reg, and to the invariants
(symmetry, positive semi-definiteness, coefficient scaling, fixed-dof rows).
The paper prints no values of F, so no pin comes from the paper itself.

Memoisation (oracle only): subdomains whose ``key`` is equal have identical
K and fixed dofs, so their K_reg^{-1} columns are shared.  This is a property
of the inputs, not of the method.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

__all__ = ["regularize", "regularized_sparse", "residual", "cholesky", "forward_substitution", "backward_substitution",
           "solve_spd", "dual_operator", "dual_operator_columns", "dual_operators", "apply_dual",
           "relative_frobenius", "NotSPDError"]


class NotSPDError(ValueError):
    pass


def regularize(K: sp.spmatrix, fixed: Sequence[int]) -> np.ndarray:
    """Dense K_reg (paper Sec. 2.2: K^+ = K_reg^{-1}, regularisation by fixing
    nodes): rows and columns of the fixed dofs are zeroed, their diagonal set
    to 1.  For a minimal fixing set the free-free block of K_reg^{-1} is the
    fixing-node generalised inverse."""
    A = sp.csr_matrix(K).toarray().astype(np.float64, copy=False)   # a fresh dense array
    f = np.asarray(fixed, dtype=np.int64)
    A[f, :] = 0.0
    A[:, f] = 0.0
    A[f, f] = 1.0
    return A


def _cholesky_unblocked(A: np.ndarray) -> np.ndarray:
    """Left-looking column Cholesky of a small dense SPD block (lower)."""
    b = A.shape[0]
    G = np.zeros_like(A)
    for j in range(b):
        d = A[j, j] - G[j, :j] @ G[j, :j]
        if not d > 0.0:
            raise NotSPDError(f"non-positive pivot {d!r} at local column {j}")
        G[j, j] = math.sqrt(d)
        G[j + 1:, j] = (A[j + 1:, j] - G[j + 1:, :j] @ G[j, :j]) / G[j, j]
    return G


def _lower_solve_small(T: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Solve T X = R for small lower-triangular T by rows."""
    X = np.empty_like(R)
    for i in range(T.shape[0]):
        X[i] = (R[i] - T[i, :i] @ X[:i]) / T[i, i]
    return X


def _upper_solve_small(U: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Solve U X = R for small upper-triangular U by rows from the bottom."""
    b = U.shape[0]
    X = np.empty_like(R)
    for i in range(b - 1, -1, -1):
        X[i] = (R[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def cholesky(A: np.ndarray, block: int = 128) -> np.ndarray:
    """Blocked left-looking dense Cholesky: A = G G^T, G lower (FP64).

    For each block column J (columns j0..j1) in turn: subtract the
    contributions of the finished columns, A[j0:, J] -= G[j0:, :j0] G[J, :j0]^T
    (one matrix product), factor the diagonal block, and solve the rows below
    against it.  Only the lower triangle is read and written.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    for j0 in range(0, n, block):
        j1 = min(j0 + block, n)
        if j0 > 0:
            A[j0:, j0:j1] -= A[j0:, :j0] @ A[j0:j1, :j0].T
        Gjj = _cholesky_unblocked(A[j0:j1, j0:j1])
        A[j0:j1, j0:j1] = Gjj
        if j1 < n:
            # panel P with P Gjj^T = A[j1:, J]  <=>  Gjj P^T = A[j1:, J]^T
            A[j1:, j0:j1] = _lower_solve_small(Gjj, A[j1:, j0:j1].T).T
    for i in range(n - 1):                       # G = lower triangle (in place: no second n x n copy)
        A[i, i + 1:] = 0.0
    return A


def forward_substitution(G: np.ndarray, R: np.ndarray, block: int = 64) -> np.ndarray:
    """Z = G^{-1} R for lower-triangular G (blocked, left-looking)."""
    n = G.shape[0]
    Z = np.empty_like(R, dtype=np.float64)
    for k0 in range(0, n, block):
        k1 = min(k0 + block, n)
        rhs = R[k0:k1] - G[k0:k1, :k0] @ Z[:k0]
        Z[k0:k1] = _lower_solve_small(G[k0:k1, k0:k1], rhs)
    return Z


def backward_substitution(G: np.ndarray, Z: np.ndarray, block: int = 64) -> np.ndarray:
    """X = G^{-T} Z for lower-triangular G (blocked, from the bottom)."""
    n = G.shape[0]
    X = np.empty_like(Z, dtype=np.float64)
    starts = list(range(0, n, block))
    for k0 in reversed(starts):
        k1 = min(k0 + block, n)
        rhs = Z[k0:k1] - G[k1:, k0:k1].T @ X[k1:]
        X[k0:k1] = _upper_solve_small(G[k0:k1, k0:k1].T, rhs)
    return X


def solve_spd(G: np.ndarray, R: np.ndarray) -> np.ndarray:
    """X = (G G^T)^{-1} R."""
    return backward_substitution(G, forward_substitution(G, R))


# ---------------------------------------------------------------------------
# error-free transformations (Dekker 1971; Knuth TAOCP vol. 2, Sec. 4.2.2)

_SPLIT = 134217729.0   # 2^27 + 1


def _two_prod(a: np.ndarray, b: np.ndarray):
    """p + e == a * b exactly (Dekker's product, Veltkamp splitting)."""
    p = a * b
    t = _SPLIT * a
    ah = t - (t - a)
    al = a - ah
    t = _SPLIT * b
    bh = t - (t - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _two_sum(a: np.ndarray, b: np.ndarray):
    """s + e == a + b exactly (Knuth's two-sum)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def regularized_sparse(K: sp.spmatrix, fixed: Sequence[int]) -> sp.csr_matrix:
    """Sparse K_reg, same definition as ``regularize``."""
    A = sp.lil_matrix(K, dtype=np.float64)
    for f in fixed:
        A[f, :] = 0.0
        A[:, f] = 0.0
        A[f, f] = 1.0
    return A.tocsr()


def residual_numpy(A: sp.csr_matrix, X: np.ndarray, R0: np.ndarray) -> np.ndarray:
    """R0 - A X with every product and sum carried in double-double, rounded
    once at the end (A sparse): per row, the stored entries in storage order,
    hi <- TwoSum(hi, p), lo <- lo + (sum error + product error)."""
    A = sp.csr_matrix(A)
    hi = np.array(R0, dtype=np.float64, copy=True)
    lo = np.zeros_like(hi)
    cnt = np.diff(A.indptr)
    for j in range(int(cnt.max()) if len(cnt) else 0):
        rows = np.nonzero(cnt > j)[0]
        idx = A.indptr[rows] + j
        a = -A.data[idx][:, None] * np.ones((1, X.shape[1]))
        p, pe = _two_prod(a, X[A.indices[idx]])
        s, se = _two_sum(hi[rows], p)
        hi[rows] = s
        lo[rows] += se + pe
    return hi + lo


_C_LIB = None


def _c_residual_lib():
    """oracle/residual.c (the loops of ``residual_numpy``), compiled once with
    gcc into oracle/_build/ (OpenMP, no fused multiply-adds); None if no C
    compiler is available."""
    global _C_LIB
    if _C_LIB is not None:
        return _C_LIB or None
    import ctypes
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "residual.c")
    out_dir = os.path.join(here, "_build")
    so = os.path.join(out_dir, "liboracle_residual.so")
    try:
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            os.makedirs(out_dir, exist_ok=True)
            tmp = so + ".%d.tmp" % os.getpid()
            subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                            src, "-o", tmp], check=True, capture_output=True)
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        vp = ctypes.c_void_p
        lib.oracle_residual.argtypes = [ctypes.c_int64, ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp]
        lib.oracle_residual.restype = None
        _C_LIB = lib
    except (OSError, subprocess.CalledProcessError):
        _C_LIB = False
    return _C_LIB or None


def build_c() -> bool:
    """Compile the oracle's C part (``residual.c``); True when it is usable."""
    return _c_residual_lib() is not None


def residual(A: sp.csr_matrix, X: np.ndarray, R0: np.ndarray) -> np.ndarray:
    """R0 - A X, error-free until one final rounding (see ``residual_numpy``);
    the same loops in C (oracle/residual.c, bit-identical results) when a C
    compiler is available, else the numpy form."""
    lib = _c_residual_lib()
    if lib is None:
        return residual_numpy(A, X, R0)
    A = sp.csr_matrix(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    R0 = np.ascontiguousarray(R0, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
        R0 = R0[:, None]
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int64)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    out = np.empty((A.shape[0], X.shape[1]))
    lo = np.empty_like(out)
    lib.oracle_residual(A.shape[0], X.shape[1], indptr.ctypes.data, indices.ctypes.data, data.ctypes.data,
                        X.ctypes.data, R0.ctypes.data, out.ctypes.data, lo.ctypes.data)
    return out[:, 0] if squeeze else out


class _Memo:
    """Per-K cache of the factor and of solved unit columns K_reg^{-1} e_d."""

    def __init__(self):
        self.G: Dict[tuple, np.ndarray] = {}
        self.cols: Dict[tuple, Dict[int, np.ndarray]] = {}


def _solve_unit_columns(sd, G: np.ndarray, dofs, refine: int) -> np.ndarray:
    """K_reg^{-1}[:, dofs]: forward/backward substitution, then ``refine``
    steps X += K_reg^{-1}(E - K_reg X) with the residual formed exactly."""
    E = np.zeros((sd.n, len(dofs)))
    E[list(dofs), np.arange(len(dofs))] = 1.0
    X = solve_spd(G, E)
    if refine:
        A = regularized_sparse(sd.K, sd.fixed)
        for _ in range(refine):
            X = X + solve_spd(G, residual(A, X, E))
    return X


def _columns(sd, dofs: np.ndarray, memo: Optional[_Memo], refine: int = 0) -> np.ndarray:
    """K_reg^{-1}[:, dofs] for the subdomain, reusing memoised columns."""
    key = getattr(sd, "key", None) if memo is not None else None
    if key is None:
        return _solve_unit_columns(sd, cholesky(regularize(sd.K, sd.fixed)), dofs, refine)
    key = (key, refine)
    if key not in memo.G:
        memo.G[key] = cholesky(regularize(sd.K, sd.fixed))
        memo.cols[key] = {}
    have = memo.cols[key]
    need = [int(d) for d in dofs if int(d) not in have]
    if need:
        X = _solve_unit_columns(sd, memo.G[key], need, refine)
        for c, d in enumerate(need):
            have[d] = X[:, c]
    return np.stack([have[int(d)] for d in dofs], axis=1)


def dual_operator(sd, memo: Optional[_Memo] = None, refine: int = 0) -> np.ndarray:
    """F = B K_reg^{-1} B^T (m x m, full symmetric), paper Eq. "localdualoperator".

    B^T may have any number of nonzeros per column; X = K_reg^{-1} B^T is
    formed from the unit columns of the distinct dofs B^T touches, with
    ``refine`` steps of iterative refinement.
    """
    Bt = sp.csc_matrix(sd.Bt)
    dofs = np.unique(Bt.indices)
    Xd = _columns(sd, dofs, memo, refine)               # n x |dofs|
    # X = K_reg^{-1} B^T = Xd @ Bt[dofs, :]
    X = Xd @ Bt[dofs, :].toarray()
    return np.asarray(Bt.T @ X)


def dual_operator_columns(sd, cols: Sequence[int], memo: Optional[_Memo] = None,
                          refine: int = 0) -> np.ndarray:
    """F[:, cols] = B K_reg^{-1} B^T[:, cols] (m x len(cols)): the same definition
    restricted to selected columns, for spot checks of large subdomains."""
    Bt = sp.csc_matrix(sd.Bt)
    sub = Bt[:, list(cols)]
    dofs = np.unique(sub.indices)
    Xd = _columns(sd, dofs, memo, refine)
    X = Xd @ sub[dofs, :].toarray()
    return np.asarray(Bt.T @ X)


def dual_operators(subdomains: Iterable, memo: Optional[_Memo] = None, refine: int = 0) -> List[np.ndarray]:
    """F_i for every subdomain, sharing K_reg^{-1} columns between equal keys."""
    memo = _Memo() if memo is None else memo
    return [dual_operator(sd, memo, refine) for sd in subdomains]


def apply_dual(Fs: Sequence[np.ndarray], lambda_maps: Sequence[np.ndarray], lam: np.ndarray,
               n_dual: int) -> np.ndarray:
    """q = sum_i B_i K_i^+ B_i^T restricted to multipliers: scatter_i(F_i lambda[map_i])
    (paper Eq. "dualop_apply_expl", accumulated over subdomains)."""
    q = np.zeros(n_dual)
    for F, mp in zip(Fs, lambda_maps):
        mp = np.asarray(mp, np.int64)
        np.add.at(q, mp, F @ lam[mp])
    return q


def relative_frobenius(A: np.ndarray, B: np.ndarray) -> float:
    """||A - B||_F / ||B||_F."""
    nb = np.linalg.norm(B)
    return float(np.linalg.norm(A - B) / (nb if nb > 0 else 1.0))
