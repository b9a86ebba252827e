"""Seeded synthetic FETI subdomain problems.

This module only *generates inputs*: structured finite-element meshes, the
subdomain stiffness matrices ``K_i`` (symmetric positive semi-definite), the
dofs that are fixed to regularise floating subdomains, and the signed-Boolean
gluing matrices ``B_i`` together with the local-to-global map of the Lagrange
multipliers.  It computes nothing of the Schur-complement method itself: no
factorisation, no triangular solve, no dual operator.  Both the CPU oracle
and the GPU library consume what it produces.

Problem family (paper Sec. 2, Eq. "fetisystemblocked"): the domain is torn
into non-overlapping subdomains; each subdomain ``i`` has a sparse SPSD
``K_i`` and a gluing matrix ``B_i`` whose rows are Lagrange multipliers.  Every
multiplier glues one dof of one subdomain to one dof of a neighbour with
entries +1 / -1 (paper Sec. 3: ``B`` has few nonzeros, on the surfaces).

Element types (the configurations use bilinear / trilinear elements):
  * 2D heat transfer, bilinear Q1 squares, 1 dof per node;
  * 3D heat transfer, trilinear hex8 cubes, 1 dof per node;
  * 3D linear elasticity, hex8 cubes, 3 dofs per node (ux, uy, uz).
Element matrices are integrated with the tensor 2-point Gauss rule, which is
exact for these elements on axis-aligned squares and cubes.

Random draws use splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) so that a seed fully determines a batch.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

__all__ = [
    "SplitMix64", "Subdomain", "Problem",
    "element_heat", "element_elasticity", "assemble_box",
    "single_heat_2d", "cube_heat_3d", "elasticity_cubes", "mixed_batch",
    "make_config", "chain_1d",
]

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream: state += golden gamma; output = mix(state)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniformly drawn from [lo, hi] (inclusive) by modulo."""
        return lo + self.next_u64() % (hi - lo + 1)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


# ----------------------------------------------------------------------------
# element matrices
# ----------------------------------------------------------------------------

_GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # on [0, 1], weights 1/2


def _shape_grads(dim: int, xi: Sequence[float]) -> np.ndarray:
    """Gradients (2**dim, dim) of the multilinear shape functions on [0,1]^dim.

    Local node ``l`` has corner bits ``(l >> d) & 1`` per axis ``d`` (x fastest).
    """
    nloc = 1 << dim
    g = np.zeros((nloc, dim))
    for l in range(nloc):
        bits = [(l >> d) & 1 for d in range(dim)]
        for d in range(dim):
            v = 1.0
            for e in range(dim):
                if e == d:
                    v *= 1.0 if bits[e] else -1.0
                else:
                    v *= xi[e] if bits[e] else (1.0 - xi[e])
            g[l, d] = v
    return g


def element_heat(dim: int, h: float, conductivity: float = 1.0) -> np.ndarray:
    """Stiffness of the Laplacian on a square/cube of side h: int grad Ni . grad Nj.

    Mapping x = h * xi gives grad_x = grad_xi / h and dV = h^dim dxi, hence the
    factor h^(dim-2).
    """
    nloc = 1 << dim
    ke = np.zeros((nloc, nloc))
    w = 0.5 ** dim
    for xi in itertools.product(_GAUSS, repeat=dim):
        g = _shape_grads(dim, xi)
        ke += w * (g @ g.T)
    return conductivity * h ** (dim - 2) * ke


def element_elasticity(h: float, E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """Hex8 isotropic linear-elasticity stiffness (24 x 24), dofs 3*l + comp."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    ke = np.zeros((24, 24))
    w = 0.125
    for xi in itertools.product(_GAUSS, repeat=3):
        g = _shape_grads(3, xi) / h          # physical gradients
        Bm = np.zeros((6, 24))
        for l in range(8):
            gx, gy, gz = g[l]
            c = 3 * l
            Bm[0, c] = gx
            Bm[1, c + 1] = gy
            Bm[2, c + 2] = gz
            Bm[3, c], Bm[3, c + 1] = gy, gx            # gamma_xy
            Bm[4, c + 1], Bm[4, c + 2] = gz, gy        # gamma_yz
            Bm[5, c], Bm[5, c + 2] = gz, gx            # gamma_xz
        ke += w * h ** 3 * (Bm.T @ D @ Bm)
    return ke


# ----------------------------------------------------------------------------
# structured-box assembly
# ----------------------------------------------------------------------------

def node_id(ix, iy, iz, nn: Tuple[int, int, int]):
    """Lexicographic node id on a (nnx, nny, nnz) node grid, x fastest."""
    return ix + nn[0] * (iy + nn[1] * iz)


def assemble_box(elems: Tuple[int, ...], ke: np.ndarray, ndpn: int) -> sp.csr_matrix:
    """Assemble a structured box of ``elems`` elements (2D or 3D) with element
    matrix ``ke`` (identical for every element) into a CSR matrix."""
    dim = len(elems)
    e3 = tuple(elems) + (0,) * (3 - dim)
    nn = tuple(e + 1 for e in e3[:dim]) + (1,) * (3 - dim)
    ex, ey, ez = np.meshgrid(*[np.arange(max(e, 1)) for e in e3], indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    if dim == 2:
        ez = np.zeros_like(ex)
    nloc = 1 << dim
    conn = np.empty((ex.size, nloc), dtype=np.int64)
    for l in range(nloc):
        bx, by, bz = l & 1, (l >> 1) & 1, (l >> 2) & 1
        conn[:, l] = node_id(ex + bx, ey + by, ez + bz, nn)
    # element dof list: ndpn * node + component
    edofs = (conn[:, :, None] * ndpn + np.arange(ndpn)[None, None, :]).reshape(ex.size, -1)
    ne = edofs.shape[1]
    rows = np.repeat(edofs, ne, axis=1).ravel()
    cols = np.tile(edofs, (1, ne)).ravel()
    vals = np.tile(ke.ravel(), ex.size)
    n = int(np.prod(nn[:dim])) * ndpn
    K = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    return K


# ----------------------------------------------------------------------------
# problem containers
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Subdomain:
    """One FETI subdomain.

    K        -- n x n SPSD stiffness (CSR, full symmetric storage), original dof order
    fixed    -- dofs fixed to regularise (rows/columns replaced by the identity)
    Bt       -- n x m gluing transpose B_i^T (CSC, entries +1/-1)
    lambda_map -- m global multiplier ids (local column j -> global dual index)
    grid     -- node-grid extents (nnx, nny, nnz); nnz == 1 in 2D
    ndpn     -- dofs per node (1 heat, 3 elasticity)
    key      -- tuple identifying K exactly (same key <=> identical K and fixed)
    """
    K: sp.csr_matrix
    fixed: np.ndarray
    Bt: sp.csc_matrix
    lambda_map: np.ndarray
    grid: Tuple[int, int, int]
    ndpn: int
    key: tuple

    @property
    def n(self) -> int:
        return self.K.shape[0]

    @property
    def m(self) -> int:
        return self.Bt.shape[1]


@dataclasses.dataclass
class Problem:
    name: str
    subdomains: List[Subdomain]
    n_dual: int
    seed: int
    description: str = ""


def _bt_from_lists(n: int, dofs: np.ndarray, signs: np.ndarray) -> sp.csc_matrix:
    m = len(dofs)
    return sp.csc_matrix((signs.astype(np.float64), (np.asarray(dofs, np.int64), np.arange(m))),
                         shape=(n, m))


_K_CACHE = {}


def _box_matrix(physics: str, elems: Tuple[int, ...], h: float, coef: float) -> sp.csr_matrix:
    key = (physics, tuple(elems), float(h), float(coef))
    if key not in _K_CACHE:
        if physics == "heat":
            ke = element_heat(len(elems), h, coef)
            _K_CACHE[key] = assemble_box(elems, ke, 1)
        elif physics == "elasticity":
            ke = element_elasticity(h, E=coef, nu=0.3)
            _K_CACHE[key] = assemble_box(elems, ke, 3)
        else:
            raise ValueError(physics)
    return _K_CACHE[key]


# ----------------------------------------------------------------------------
# configuration 1: one 2D heat subdomain
# ----------------------------------------------------------------------------

def single_heat_2d(k: int = 16, drop_fixed_corner: bool = False) -> Problem:
    """k x k Q1 squares on the unit square, corner node (0,0) fixed, B^T selects
    every boundary node (+1), columns in lexicographic node order."""
    h = 1.0 / k
    K = _box_matrix("heat", (k, k), h, 1.0)
    nn = (k + 1, k + 1, 1)
    ids = []
    for iy in range(k + 1):
        for ix in range(k + 1):
            if ix in (0, k) or iy in (0, k):
                ids.append(node_id(ix, iy, 0, nn))
    ids = np.array(ids, dtype=np.int64)
    if drop_fixed_corner:
        ids = ids[ids != 0]
    Bt = _bt_from_lists(K.shape[0], ids, np.ones(len(ids)))
    sd = Subdomain(K=K, fixed=np.array([0], np.int64), Bt=Bt,
                   lambda_map=np.arange(len(ids), dtype=np.int64), grid=nn, ndpn=1,
                   key=("heat2d", k, 1.0, (0,)))
    return Problem("heat2d_single", [sd], len(ids), 0,
                   f"2D heat, {k}x{k} Q1, corner fixed, {len(ids)} boundary multipliers")


# ----------------------------------------------------------------------------
# configuration 2: conforming 3D heat cube split into s^3 subdomains
# ----------------------------------------------------------------------------

def cube_heat_3d(parts: int = 4, k: int = 16, coef_seed: Optional[int] = None) -> Problem:
    """Unit cube split into parts^3 subdomains of k^3 hex8 elements (h = 1/(parts*k)).

    Every subdomain is floating: local node (0,0,0) is fixed.  Gluing is
    non-redundant: a global node shared by the sorted subdomains s_1 < ... < s_q
    gets multipliers (s_a, s_a+1), a = 1..q-1, with +1 on s_a and -1 on s_a+1.
    Global multiplier ids follow (global node lexicographic, pair index).
    With ``coef_seed`` each subdomain gets a conductivity drawn log-uniformly
    from [1/2, 2] (otherwise 1).
    """
    h = 1.0 / (parts * k)
    G = parts * k + 1                      # global nodes per axis
    nsub = parts ** 3
    coefs = np.ones(nsub)
    if coef_seed is not None:
        rng = SplitMix64(coef_seed)
        coefs = np.array([2.0 ** (2.0 * rng.uniform() - 1.0) for _ in range(nsub)])

    def owners(g):
        if g % k == 0 and 0 < g < G - 1:
            return (g // k - 1, g // k)
        return (min(g // k, parts - 1),)

    own = [owners(g) for g in range(G)]
    nn_loc = (k + 1, k + 1, k + 1)
    cols = [[] for _ in range(nsub)]    # (global multiplier id, local dof, sign)
    mult = 0
    for gz in range(G):
        oz = own[gz]
        for gy in range(G):
            oy = own[gy]
            for gx in range(G):
                ox = own[gx]
                if len(ox) * len(oy) * len(oz) < 2:
                    continue
                subs = sorted(a + parts * (b + parts * c) for c in oz for b in oy for a in ox)
                for s0, s1 in zip(subs[:-1], subs[1:]):
                    for s, sign in ((s0, 1.0), (s1, -1.0)):
                        a, b, c = s % parts, (s // parts) % parts, s // (parts * parts)
                        loc = node_id(gx - a * k, gy - b * k, gz - c * k, nn_loc)
                        cols[s].append((mult, loc, sign))
                    mult += 1
    subs_out = []
    for s in range(nsub):
        K = _box_matrix("heat", (k, k, k), h, float(coefs[s]))
        c = np.array(cols[s], dtype=np.float64).reshape(-1, 3)
        order = np.argsort(c[:, 0], kind="stable")
        c = c[order]
        Bt = _bt_from_lists(K.shape[0], c[:, 1].astype(np.int64), c[:, 2])
        subs_out.append(Subdomain(K=K, fixed=np.array([0], np.int64), Bt=Bt,
                                  lambda_map=c[:, 0].astype(np.int64), grid=nn_loc, ndpn=1,
                                  key=("heat3d", k, h, float(coefs[s]), (0,))))
    return Problem(f"heat3d_cube_{parts}x{k}", subs_out, mult, coef_seed or 0,
                   f"3D heat, {parts}^3 subdomains of {k}^3 hex8, non-redundant gluing")


# ----------------------------------------------------------------------------
# configurations 3 and 5: uneven subdomains on a lattice
# ----------------------------------------------------------------------------

def _elasticity_fixed(k: int) -> np.ndarray:
    """Minimal fixing of the 6 rigid-body modes of a k^3 hex8 cube:
    node (0,0,0) in x,y,z; node (k,0,0) in y,z; node (0,k,0) in z."""
    nn = (k + 1, k + 1, k + 1)
    n0 = node_id(0, 0, 0, nn)
    n1 = node_id(k, 0, 0, nn)
    n2 = node_id(0, k, 0, nn)
    return np.array([3 * n0, 3 * n0 + 1, 3 * n0 + 2, 3 * n1 + 1, 3 * n1 + 2, 3 * n2 + 2], np.int64)


def _lattice_gluing(dims: Tuple[int, ...], ks: List[int], ndpn: int):
    """Gluing on a lattice of uneven square/cube subdomains (one per lattice cell).

    Across each lattice face (edge in 2D) between neighbours a, b with k_a <= k_b
    there are (k_a+1)^(d-1) face nodes of a, each matched to b's face node at
    round(u * k_b / k_a) (injective since k_b >= k_a); one multiplier per
    matched node and component, +1 on the lower subdomain id.  A node on
    several glued faces gets one multiplier per face.  Faces are visited in
    (axis, lower cell id) order, nodes lexicographically on the face.
    """
    d = len(dims)
    ncell = int(np.prod(dims))
    cols = [[] for _ in range(ncell)]
    mult = 0

    def cell_id(c):
        r, st = 0, 1
        for a in range(d):
            r += c[a] * st
            st *= dims[a]
        return r

    def local_node(k, coords):
        nn = (k + 1,) * d + (1,) * (3 - d)
        x = list(coords) + [0] * (3 - d)
        return node_id(x[0], x[1], x[2], nn)

    for axis in range(d):
        for cell in itertools.product(*[range(n) for n in dims[::-1]]):
            c = cell[::-1]
            if c[axis] + 1 >= dims[axis]:
                continue
            nb = list(c)
            nb[axis] += 1
            ia, ib = cell_id(c), cell_id(nb)
            ka, kb = ks[ia], ks[ib]
            # face coordinates on the coarser side
            small, large = (ia, ib) if ka <= kb else (ib, ia)
            ks_, kl_ = ks[small], ks[large]
            other = [a for a in range(d) if a != axis]
            for uv in itertools.product(*[range(ks_ + 1) for _ in other]):
                cs = [0] * d
                cl = [0] * d
                for a, u in zip(other, uv):
                    cs[a] = u
                    cl[a] = int(round(u * kl_ / ks_))
                # the lower cell touches the face at its max coordinate
                if small == ia:
                    cs[axis], cl[axis] = ks_, 0
                else:
                    cs[axis], cl[axis] = 0, kl_
                ns_, nl_ = local_node(ks_, cs), local_node(kl_, cl)
                for comp in range(ndpn):
                    sa = 1.0 if small < large else -1.0
                    cols[small].append((mult, ndpn * ns_ + comp, sa))
                    cols[large].append((mult, ndpn * nl_ + comp, -sa))
                    mult += 1
    return cols, mult


def _lattice_problem(name, physics, dims, ks, seed, desc) -> Problem:
    d = len(dims)
    ndpn = 3 if physics == "elasticity" else 1
    cols, nmult = _lattice_gluing(dims, ks, ndpn)
    subs = []
    for i, k in enumerate(ks):
        K = _box_matrix(physics, (k,) * d, 1.0 / k, 1.0)
        fixed = _elasticity_fixed(k) if physics == "elasticity" else np.array([0], np.int64)
        c = np.array(cols[i], dtype=np.float64).reshape(-1, 3)
        c = c[np.argsort(c[:, 0], kind="stable")]
        Bt = _bt_from_lists(K.shape[0], c[:, 1].astype(np.int64), c[:, 2])
        nn = (k + 1,) * d + (1,) * (3 - d)
        subs.append(Subdomain(K=K, fixed=fixed, Bt=Bt, lambda_map=c[:, 0].astype(np.int64),
                              grid=nn, ndpn=ndpn, key=(physics, d, k, tuple(fixed))))
    return Problem(name, subs, nmult, seed, desc)


def elasticity_cubes(lattice=(8, 8, 8), kmin: int = 8, kmax: int = 16, seed: int = 0) -> Problem:
    """Uneven 3D elasticity cubes (E=1, nu=0.3, unit cube each, h = 1/k)."""
    rng = SplitMix64(seed)
    ncell = int(np.prod(lattice))
    ks = [rng.randint(kmin, kmax) for _ in range(ncell)]
    return _lattice_problem(f"elasticity_{'x'.join(map(str, lattice))}", "elasticity",
                            lattice, ks, seed,
                            f"3D elasticity cubes, k in [{kmin},{kmax}], lattice {lattice}")


def mixed_batch(lat2d=(32, 32), k2d=(32, 96), lat3d=(16, 8, 8), k3d=(8, 20), seed: int = 0) -> Problem:
    """Half 2D heat squares, half 3D elasticity cubes; sizes drawn from one
    splitmix64 stream alternating 2D/3D by draw index."""
    rng = SplitMix64(seed)
    n2, n3 = int(np.prod(lat2d)), int(np.prod(lat3d))
    ks2, ks3 = [], []
    while len(ks2) < n2 or len(ks3) < n3:
        if len(ks2) < n2:
            ks2.append(rng.randint(*k2d))
        if len(ks3) < n3:
            ks3.append(rng.randint(*k3d))
    p2 = _lattice_problem("heat2d", "heat", lat2d, ks2, seed, "")
    p3 = _lattice_problem("elasticity", "elasticity", lat3d, ks3, seed, "")
    for sd in p3.subdomains:                    # two independent dual spaces, stacked
        sd.lambda_map = sd.lambda_map + p2.n_dual
    return Problem("mixed", p2.subdomains + p3.subdomains, p2.n_dual + p3.n_dual, seed,
                   "mixed 2D heat + 3D elasticity batch")


def make_config(idx: int, seed: int = 0, **kw) -> Problem:
    """The five workload configurations (1-based index)."""
    if idx == 1:
        return single_heat_2d(16, **kw)
    if idx in (2, 4):
        return cube_heat_3d(4, 16, **kw)
    if idx == 3:
        return elasticity_cubes((8, 8, 8), 8, 16, seed)
    if idx == 5:
        return mixed_batch(seed=seed)
    raise ValueError(idx)


# ----------------------------------------------------------------------------
# a 1D chain (used by closed-form checks)
# ----------------------------------------------------------------------------

def chain_1d(nel: int, select: Sequence[int], signs: Optional[Sequence[float]] = None) -> Subdomain:
    """Linear elements on [0,1], nodes 0..nel, h = 1/nel, unit conductivity,
    node 0 fixed; B^T selects the listed nodes."""
    h = 1.0 / nel
    n = nel + 1
    main = np.full(n, 2.0 / h)
    main[0] = main[-1] = 1.0 / h
    off = np.full(n - 1, -1.0 / h)
    K = sp.diags([off, main, off], [-1, 0, 1], format="csr")
    sel = np.asarray(select, np.int64)
    sg = np.ones(len(sel)) if signs is None else np.asarray(signs, np.float64)
    return Subdomain(K=K, fixed=np.array([0], np.int64), Bt=_bt_from_lists(n, sel, sg),
                     lambda_map=np.arange(len(sel), dtype=np.int64), grid=(n, 1, 1), ndpn=1,
                     key=("chain", nel))
