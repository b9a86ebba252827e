"""Host-side input production: fill-reducing ordering and sparse Cholesky.

The Schur-complement assembly starts from a *given* sparse Cholesky factor L
of the regularised subdomain matrix (paper Sec. 2.2 and Sec. 3: the input is
B^T together with L, both in the fill-reducing order of the symbolic
factorisation).  This module produces that input on the CPU:

  * ``nested_dissection`` -- geometric nested dissection on the structured
    node grid (bisect the longest axis, separator plane ordered last, recurse
    down to small leaf boxes; the dofs of a node stay contiguous).  The paper
    uses METIS for this step; on structured grids geometric dissection gives
    the same kind of ordering without a graph partitioner;
  * ``factorize`` -- the native host Cholesky (libscfactor.so) on
    P K_reg P^T, with the etree postorder composed into P;
  * ``factorize_problem`` -- the above for every subdomain of a batch, with
    identical (K, fixed) pairs factorised once (the factor is an input; the
    GPU library still reads every subdomain's values separately).
"""
from __future__ import annotations

import ctypes
import dataclasses
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

from . import _native


def nested_dissection(grid: Tuple[int, int, int], ndpn: int = 1, leaf: int = 8) -> np.ndarray:
    """Dof permutation new -> old for a lexicographic (x fastest) node grid."""
    nx, ny, nz = grid
    order: List[np.ndarray] = []

    def box_nodes(lo, hi):
        xs, ys, zs = (np.arange(lo[a], hi[a]) for a in range(3))
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        return (X + nx * (Y + ny * Z)).ravel()

    stack = [((0, 0, 0), (nx, ny, nz), False)]
    # iterative post-order: left box, right box, then separator
    out: List[np.ndarray] = []

    def rec(lo, hi):
        ext = [hi[a] - lo[a] for a in range(3)]
        cnt = ext[0] * ext[1] * ext[2]
        if cnt == 0:
            return
        if cnt <= leaf or max(ext) < 3:
            out.append(box_nodes(lo, hi))
            return
        ax = int(np.argmax(ext))
        mid = lo[ax] + ext[ax] // 2
        lhi = list(hi); lhi[ax] = mid
        rlo = list(lo); rlo[ax] = mid + 1
        slo = list(lo); slo[ax] = mid
        shi = list(hi); shi[ax] = mid + 1
        rec(tuple(lo), tuple(lhi))
        rec(tuple(rlo), tuple(hi))
        out.append(box_nodes(tuple(slo), tuple(shi)))

    rec((0, 0, 0), (nx, ny, nz))
    nodes = np.concatenate(out)
    assert len(nodes) == nx * ny * nz
    return (nodes[:, None] * ndpn + np.arange(ndpn)[None, :]).ravel().astype(np.int32)


@dataclasses.dataclass
class HostFactor:
    """L (CSC lower, rows ascending, diagonal first) of P K_reg P^T and P."""
    n: int
    colptr: np.ndarray   # int64 [n+1]
    rowind: np.ndarray   # int32 [nnz]
    values: np.ndarray   # float64 [nnz]
    perm: np.ndarray     # int32 [n], new -> old

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    @property
    def iperm(self) -> np.ndarray:
        ip = np.empty(self.n, np.int32)
        ip[self.perm] = np.arange(self.n, dtype=np.int32)
        return ip


def factorize(K: sp.spmatrix, fixed: Sequence[int], perm: Optional[np.ndarray] = None,
              postorder: bool = True) -> HostFactor:
    lib = _native.factor_lib()
    Kc = sp.csc_matrix(K)
    Kc.sort_indices()
    n = Kc.shape[0]
    cp = np.ascontiguousarray(Kc.indptr, dtype=np.int64)
    ri = np.ascontiguousarray(Kc.indices, dtype=np.int32)
    va = np.ascontiguousarray(Kc.data, dtype=np.float64)
    fx = np.ascontiguousarray(np.asarray(fixed), dtype=np.int32)
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = lib.scf_factorize(n, cp.ctypes.data, ri.ctypes.data, va.ctypes.data, len(fx),
                           fx.ctypes.data if len(fx) else None,
                           pm.ctypes.data if pm is not None else None, int(postorder), ctypes.byref(h))
    if rc != 0:
        raise RuntimeError(f"scf_factorize failed with code {rc}")
    try:
        nnz = lib.scf_nnz(h)
        out = HostFactor(n, np.empty(n + 1, np.int64), np.empty(nnz, np.int32),
                         np.empty(nnz, np.float64), np.empty(n, np.int32))
        lib.scf_export(h, out.colptr.ctypes.data, out.rowind.ctypes.data, out.values.ctypes.data,
                       out.perm.ctypes.data)
    finally:
        lib.scf_free(h)
    return out


def solve_LLt(L: HostFactor, b: np.ndarray) -> np.ndarray:
    """x = L^-T L^-1 b in L's ordering (scf_solve: two sparse triangular
    solves on the host)."""
    b = np.ascontiguousarray(b, np.float64)
    assert b.shape == (L.n,)
    x = np.empty(L.n)
    cp = np.ascontiguousarray(L.colptr, np.int64)
    ri = np.ascontiguousarray(L.rowind, np.int32)
    va = np.ascontiguousarray(L.values, np.float64)
    rc = _native.factor_lib().scf_solve(L.n, cp.ctypes.data, ri.ctypes.data, va.ctypes.data, b.ctypes.data,
                                        x.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"scf_solve failed with code {rc}")
    return x


class SymbolicFactor:
    """The symbolic stage alone (scf_analyze): the ordering and L's pattern
    for K's pattern, kept so that ``numeric`` runs only the numeric stage
    (scf_numeric) for any values on that pattern (paper Sec. 2.2)."""

    def __init__(self, K: sp.spmatrix, fixed: Sequence[int], perm: Optional[np.ndarray] = None,
                 postorder: bool = True):
        lib = _native.factor_lib()
        Kc = sp.csc_matrix(K)
        Kc.sort_indices()
        self.n = Kc.shape[0]
        self._cp = np.ascontiguousarray(Kc.indptr, dtype=np.int64)
        self._ri = np.ascontiguousarray(Kc.indices, dtype=np.int32)
        fx = np.ascontiguousarray(np.asarray(fixed), dtype=np.int32)
        pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        h = ctypes.c_void_p()
        rc = lib.scf_analyze(self.n, self._cp.ctypes.data, self._ri.ctypes.data, len(fx),
                             fx.ctypes.data if len(fx) else None, pm.ctypes.data if pm is not None else None,
                             int(postorder), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"scf_analyze failed with code {rc}")
        self._h = h
        nnz = lib.scf_nnz(h)
        self.colptr = np.empty(self.n + 1, np.int64)
        self.rowind = np.empty(nnz, np.int32)
        self.perm = np.empty(self.n, np.int32)
        lib.scf_export(h, self.colptr.ctypes.data, self.rowind.ctypes.data, None, self.perm.ctypes.data)

    def numeric(self, K: sp.spmatrix) -> HostFactor:
        """L for K's values; K must have the analysed pattern."""
        Kc = sp.csc_matrix(K)
        Kc.sort_indices()
        if not (np.array_equal(Kc.indptr, self._cp) and np.array_equal(Kc.indices, self._ri)):
            raise ValueError("K does not have the analysed pattern")
        va = np.ascontiguousarray(Kc.data, dtype=np.float64)
        values = np.empty(len(self.rowind), np.float64)
        rc = _native.factor_lib().scf_numeric(self._h, va.ctypes.data, values.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"scf_numeric failed with code {rc}")
        return HostFactor(self.n, self.colptr.copy(), self.rowind.copy(), values, self.perm.copy())

    def __del__(self):
        try:
            h = getattr(self, "_h", None)
            if h is not None and h.value:
                _native.factor_lib().scf_free(h)
                self._h = None
        except Exception:
            pass


@dataclasses.dataclass
class FactoredSubdomain:
    """Library input for one subdomain: L in the fill-reducing order and B^T
    with rows renumbered into that order (columns untouched)."""
    L: HostFactor
    bt_colptr: np.ndarray   # int32 [m+1]
    bt_rowind: np.ndarray   # int32 [nnz(B^T)], rows in L's ordering
    bt_sign: np.ndarray     # int8  [nnz(B^T)]
    lambda_map: np.ndarray  # int32 [m]
    bt_val: Optional[np.ndarray] = None   # float64 [nnz(B^T)]: general values in place of bt_sign

    @property
    def n(self) -> int:
        return self.L.n

    @property
    def m(self) -> int:
        return len(self.bt_colptr) - 1


def permute_bt(sd, L: HostFactor) -> FactoredSubdomain:
    Bt = sp.csc_matrix(sd.Bt)
    ip = L.iperm
    rows = ip[Bt.indices]
    cp = Bt.indptr.astype(np.int32)
    # rows ascending within each column
    ri = rows.astype(np.int32).copy()
    sg = np.sign(Bt.data).astype(np.int8)
    for j in range(Bt.shape[1]):
        a, b = cp[j], cp[j + 1]
        if b - a > 1:
            o = np.argsort(ri[a:b], kind="stable")
            ri[a:b] = ri[a:b][o]
            sg[a:b] = sg[a:b][o]
    return FactoredSubdomain(L, cp, ri, sg, np.asarray(sd.lambda_map, np.int32))


class _ApplySub(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("L_colptr", ctypes.c_void_p),
                ("L_rowind", ctypes.c_void_p), ("L_val", ctypes.c_void_p), ("Bt_colptr", ctypes.c_void_p),
                ("Bt_rowind", ctypes.c_void_p), ("Bt_sign", ctypes.c_void_p), ("lambda_map", ctypes.c_void_p)]


class ImplicitApply:
    """Host implicit application q = sum_i B_i L_i^-T L_i^-1 B_i^T lambda_i
    (paper Eq. "dualop_apply_impl"), the per-iteration alternative to the
    explicit F*lambda.  planned=True (default) makes the supernodal plan once
    (scf_implicit_plan) and runs it per call (scf_implicit_run);
    planned=False runs the column-by-column scf_implicit_apply."""

    def __init__(self, subdomains: Sequence[FactoredSubdomain], n_dual: int, planned: bool = True):
        self.lib = _native.factor_lib()
        self.n_dual = int(n_dual)
        self._keep = []
        self.arr = (_ApplySub * max(1, len(subdomains)))()
        for i, fs in enumerate(subdomains):
            a = [np.ascontiguousarray(fs.L.colptr, np.int64), np.ascontiguousarray(fs.L.rowind, np.int32),
                 np.ascontiguousarray(fs.L.values, np.float64), np.ascontiguousarray(fs.bt_colptr, np.int32),
                 np.ascontiguousarray(fs.bt_rowind, np.int32), np.ascontiguousarray(fs.bt_sign, np.int8),
                 np.ascontiguousarray(fs.lambda_map, np.int32)]
            self._keep += a
            s = self.arr[i]
            s.n, s.m = fs.n, fs.m
            s.L_colptr, s.L_rowind, s.L_val, s.Bt_colptr, s.Bt_rowind, s.Bt_sign, s.lambda_map = \
                [x.ctypes.data if x.size else None for x in a]
        self.nsub = len(subdomains)
        self._plan = None
        if planned:
            h = ctypes.c_void_p()
            rc = self.lib.scf_implicit_plan(self.nsub, self.arr, self.n_dual, ctypes.byref(h))
            if rc != 0:
                raise RuntimeError(f"scf_implicit_plan failed ({rc})")
            self._plan = h

    def __call__(self, lam: np.ndarray, threads: int = 0) -> np.ndarray:
        lam = np.ascontiguousarray(lam, np.float64)
        q = np.empty(self.n_dual)
        if self._plan is not None:
            rc = self.lib.scf_implicit_run(self._plan, lam.ctypes.data, q.ctypes.data, threads)
        else:
            rc = self.lib.scf_implicit_apply(self.nsub, self.arr, self.n_dual, lam.ctypes.data, q.ctypes.data,
                                             threads)
        if rc != 0:
            raise RuntimeError(f"host implicit apply failed ({rc})")
        return q

    def __del__(self):
        try:
            h = getattr(self, "_plan", None)
            if h is not None and h.value:
                self.lib.scf_implicit_free(h)
                self._plan = None
        except Exception:
            pass


def factorize_problem(subdomains, threads: int = 0, leaf: int = 8) -> List[FactoredSubdomain]:
    """Order and factorise every subdomain (identical keys factorised once)."""
    keys: Dict[object, int] = {}
    uniq = []
    for sd in subdomains:
        k = sd.key if sd.key is not None else id(sd)
        if k not in keys:
            keys[k] = len(uniq)
            uniq.append(sd)

    def work(sd):
        p = nested_dissection(sd.grid, sd.ndpn, leaf)
        return factorize(sd.K, sd.fixed, p, postorder=True)

    if threads == 1 or len(uniq) == 1:
        facs = [work(sd) for sd in uniq]
    else:
        # largest first (the factorisation cost grows like n^2 in 3D, n^1.5 in 2D), so that
        # the biggest subdomains do not start last and set the time of the whole batch
        cost = [sd.K.shape[0] ** (2.0 if sd.grid[2] > 1 else 1.5) for sd in uniq]
        order = sorted(range(len(uniq)), key=lambda j: -cost[j])
        facs = [None] * len(uniq)
        with ThreadPoolExecutor(max_workers=threads or None) as ex:
            for j, fac in zip(order, ex.map(work, [uniq[j] for j in order])):
                facs[j] = fac
    out = []
    for sd in subdomains:
        k = sd.key if sd.key is not None else id(sd)
        out.append(permute_bt(sd, facs[keys[k]]))
    return out
