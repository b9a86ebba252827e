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

__all__ = ["regularize", "cholesky", "forward_substitution", "backward_substitution",
           "solve_spd", "dual_operator", "dual_operator_columns", "dual_operators", "apply_dual",
           "relative_frobenius", "NotSPDError"]


class NotSPDError(ValueError):
    pass


def regularize(K: sp.spmatrix, fixed: Sequence[int]) -> np.ndarray:
    """Dense K_reg (paper Sec. 2.2: K^+ = K_reg^{-1}, regularisation by fixing
    nodes): rows and columns of the fixed dofs are zeroed, their diagonal set
    to 1.  For a minimal fixing set the free-free block of K_reg^{-1} is the
    fixing-node generalised inverse."""
    A = np.asarray(K.todense(), dtype=np.float64).copy()
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


def cholesky(A: np.ndarray, block: int = 64) -> np.ndarray:
    """Blocked right-looking dense Cholesky: A = G G^T, G lower (FP64).

    For each diagonal block: factor it, solve the panel below against it,
    subtract the panel's outer product from the trailing matrix.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    for k0 in range(0, n, block):
        k1 = min(k0 + block, n)
        Gkk = _cholesky_unblocked(A[k0:k1, k0:k1])
        A[k0:k1, k0:k1] = Gkk
        if k1 < n:
            # panel P with P Gkk^T = A[k1:, k0:k1]  <=>  Gkk P^T = A[k1:, k0:k1]^T
            P = _lower_solve_small(Gkk, A[k1:, k0:k1].T).T
            A[k1:, k0:k1] = P
            A[k1:, k1:] -= P @ P.T
    return np.tril(A)


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


class _Memo:
    """Per-K cache of the factor and of solved unit columns K_reg^{-1} e_d."""

    def __init__(self):
        self.G: Dict[tuple, np.ndarray] = {}
        self.cols: Dict[tuple, Dict[int, np.ndarray]] = {}


def _columns(sd, dofs: np.ndarray, memo: Optional[_Memo]) -> np.ndarray:
    """K_reg^{-1}[:, dofs] for the subdomain, reusing memoised columns."""
    key = getattr(sd, "key", None) if memo is not None else None
    if key is None:
        G = cholesky(regularize(sd.K, sd.fixed))
        E = np.zeros((sd.n, len(dofs)))
        E[dofs, np.arange(len(dofs))] = 1.0
        return solve_spd(G, E)
    if key not in memo.G:
        memo.G[key] = cholesky(regularize(sd.K, sd.fixed))
        memo.cols[key] = {}
    have = memo.cols[key]
    need = [int(d) for d in dofs if int(d) not in have]
    if need:
        E = np.zeros((sd.n, len(need)))
        E[need, np.arange(len(need))] = 1.0
        X = solve_spd(memo.G[key], E)
        for c, d in enumerate(need):
            have[d] = X[:, c]
    return np.stack([have[int(d)] for d in dofs], axis=1)


def dual_operator(sd, memo: Optional[_Memo] = None) -> np.ndarray:
    """F = B K_reg^{-1} B^T (m x m, full symmetric), paper Eq. "localdualoperator".

    B^T may have any number of nonzeros per column; X = K_reg^{-1} B^T is
    formed from the unit columns of the distinct dofs B^T touches.
    """
    Bt = sp.csc_matrix(sd.Bt)
    dofs = np.unique(Bt.indices)
    Xd = _columns(sd, dofs, memo)                       # n x |dofs|
    # X = K_reg^{-1} B^T = Xd @ Bt[dofs, :]
    X = Xd @ Bt[dofs, :].toarray()
    return np.asarray(Bt.T @ X)


def dual_operator_columns(sd, cols: Sequence[int], memo: Optional[_Memo] = None) -> np.ndarray:
    """F[:, cols] = B K_reg^{-1} B^T[:, cols] (m x len(cols)): the same definition
    restricted to selected columns, for spot checks of large subdomains."""
    Bt = sp.csc_matrix(sd.Bt)
    sub = Bt[:, list(cols)]
    dofs = np.unique(sub.indices)
    Xd = _columns(sd, dofs, memo)
    X = Xd @ sub[dofs, :].toarray()
    return np.asarray(Bt.T @ X)


def dual_operators(subdomains: Iterable, memo: Optional[_Memo] = None) -> List[np.ndarray]:
    """F_i for every subdomain, sharing K_reg^{-1} columns between equal keys."""
    memo = _Memo() if memo is None else memo
    return [dual_operator(sd, memo) for sd in subdomains]


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
