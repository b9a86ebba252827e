"""CPU-side checks of the C ABI: the library loads and exports every declared
symbol; sc_plan validates its inputs; the exported plan keeps every kernel
address in bounds and, replayed on the CPU, reproduces the oracle's F."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from paper_2509_21037_gb300 import _native, abi, host, implicit, sc

import implicit_emulator as ie
import plan_emulator as pe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sc\w*)\s*\(", src, flags=re.M))


@pytest.mark.parametrize("header,loader", [("sc.h", _native.sc_lib), ("sc_dense.h", _native.dense_lib),
                                           ("sc_factor.h", _native.factor_lib), ("sc_implicit.h", _native.sc_lib),
                                           ("sc_pipeline.h", _native.pipe_lib),
                                           ("sc_probe.h", _native.sc_lib), ("sc_mlp.h", _native.sc_lib)])
def test_library_exports_every_declared_symbol(header, loader):
    names = _declared(header)
    assert names, header
    lib = loader()
    for n in names:
        assert hasattr(lib, n), f"{n} declared in {header} but not exported"


def test_binding_covers_header():
    assert _declared("sc.h") == set(abi.SC_SYMBOLS)
    assert _declared("sc_dense.h") == set(abi.DENSE_SYMBOLS)
    assert _declared("sc_implicit.h") == set(abi.IMPLICIT_SYMBOLS)
    assert _declared("sc_pipeline.h") == set(abi.PIPELINE_SYMBOLS)
    assert _declared("sc_probe.h") == set(abi.PROBE_SYMBOLS)


def _plan_raw(descs, n_dual):
    lib = _native.sc_lib()
    h = ctypes.c_void_p()
    arr = (abi.SubdomainDesc * max(1, len(descs)))(*descs)
    st = lib.sc_plan(ctypes.byref(h), len(descs), arr, n_dual, None)
    msg = lib.sc_last_error(h).decode() if h.value else ""
    if h.value:
        lib.sc_destroy(h)
    return st, msg


def _desc_from(fs, keep, **over):
    arrs = dict(colptr=fs.L.colptr.copy(), rowind=fs.L.rowind.copy(), btc=fs.bt_colptr.copy(),
                btr=fs.bt_rowind.copy(), sign=fs.bt_sign.copy(), lam=fs.lambda_map.copy())
    arrs.update(over)
    keep.append(arrs)
    d = abi.SubdomainDesc()
    d.n = over.get("n", fs.n)
    d.m = over.get("m", fs.m)
    d.L_colptr = arrs["colptr"].ctypes.data
    d.L_rowind = arrs["rowind"].ctypes.data
    d.Bt_colptr = arrs["btc"].ctypes.data
    d.Bt_rowind = arrs["btr"].ctypes.data
    d.Bt_sign = arrs["sign"].ctypes.data
    d.lambda_map = arrs["lam"].ctypes.data
    return d


@pytest.fixture(scope="module")
def cfg1():
    prob = synth.make_config(1)
    return prob, host.factorize_problem(prob.subdomains)


def test_plan_accepts_valid(cfg1):
    prob, fs = cfg1
    keep = []
    st, msg = _plan_raw([_desc_from(fs[0], keep)], prob.n_dual)
    assert st == abi.SC_OK, msg


@pytest.mark.parametrize("case", ["diag_not_first", "row_out_of_range", "bad_sign", "bt_unsorted",
                                  "lambda_out_of_range", "negative_m"])
def test_plan_rejects_invalid(cfg1, case):
    prob, fs = cfg1
    f = fs[0]
    keep = []
    if case == "diag_not_first":
        ri = f.L.rowind.copy()
        a = f.L.colptr[5]
        ri[a], ri[a + 1] = ri[a + 1], ri[a]
        d = _desc_from(f, keep, rowind=ri)
    elif case == "row_out_of_range":
        ri = f.L.rowind.copy()
        ri[f.L.colptr[3] + 1] = f.n + 7
        d = _desc_from(f, keep, rowind=ri)
    elif case == "bad_sign":
        sg = f.bt_sign.copy()
        sg[0] = 2
        d = _desc_from(f, keep, sign=sg)
    elif case == "bt_unsorted":
        # column 0 with two rows in descending order
        btc = f.bt_colptr.copy()
        btc[1:] += 1
        btr = np.concatenate([[f.bt_rowind[0] + 1, f.bt_rowind[0]], f.bt_rowind[1:]]).astype(np.int32)
        sg = np.concatenate([[1, 1], f.bt_sign[1:]]).astype(np.int8)
        d = _desc_from(f, keep, btc=btc, btr=btr, sign=sg)
    elif case == "lambda_out_of_range":
        lam = f.lambda_map.copy()
        lam[3] = prob.n_dual
        d = _desc_from(f, keep, lam=lam)
    else:
        d = _desc_from(f, keep, m=-1)
    st, msg = _plan_raw([d], prob.n_dual)
    assert st == abi.SC_ERR_INVALID_ARG and msg


def test_empty_batch_and_empty_subdomain():
    st, _ = _plan_raw([], 0)
    assert st == abi.SC_OK
    d = abi.SubdomainDesc()
    cp = np.array([0, 1, 2], np.int64)
    ri = np.array([0, 1], np.int32)
    btc = np.array([0], np.int32)
    d.n, d.m = 2, 0
    d.L_colptr, d.L_rowind, d.Bt_colptr = cp.ctypes.data, ri.ctypes.data, btc.ctypes.data
    st, msg = _plan_raw([d], 0)
    assert st == abi.SC_OK, msg


def edge_batch():
    """cube_heat_3d(2, 5) with subdomain 0 unglued (m = 0) and subdomains 1,
    2, 3 cut to 64, 32 and 1 multipliers (exact tile multiples and a single
    column); the others keep their ragged 91..102."""
    prob = synth.cube_heat_3d(2, 5)
    subs = list(prob.subdomains)
    for i, m in ((0, 0), (1, 64), (2, 32), (3, 1)):
        sd = subs[i]
        subs[i] = synth.Subdomain(K=sd.K, fixed=sd.fixed, Bt=sp.csc_matrix(sd.Bt)[:, :m],
                                  lambda_map=np.asarray(sd.lambda_map)[:m], grid=sd.grid, ndpn=sd.ndpn, key=None)
    return synth.Problem(name="edge_batch", subdomains=subs, n_dual=prob.n_dual, seed=0, description="edge cases")


def _cases():
    yield "config1", synth.make_config(1)
    yield "edge_batch", edge_batch()
    yield "cube_2x5", synth.cube_heat_3d(2, 5)
    yield "cube_coef", synth.cube_heat_3d(2, 3, coef_seed=4)
    yield "elast", synth.elasticity_cubes((2, 1, 1), 2, 3, seed=1)


@pytest.mark.parametrize("name,prob", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_plan_emulation_matches_oracle(name, prob):
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual)
    T = pe.export_plan(plan)
    pe.check_bounds(T, plan.sizes, plan.stats)
    F = pe.emulate_assembly(T, plan.sizes, plan.stats, sc.concat_L_values(fs))
    assert not np.isnan(F).any(), "F entries left unwritten"
    Fo = oracle.dual_operators(prob.subdomains)
    for i in range(len(fs)):
        assert oracle.relative_frobenius(pe.export_dense(T, F, i), Fo[i]) <= 1e-12


@pytest.mark.parametrize("name,prob", [c for c in _cases() if c[0] != "config1"] +
                         [("mixed", synth.mixed_batch(lat2d=(2, 2), k2d=(6, 40), lat3d=(2, 1, 1), k3d=(2, 6), seed=3))],
                         ids=lambda x: x if isinstance(x, str) else "")
def test_tile_plan_emulation_matches_oracle(name, prob):
    """Split-precision subdomains with the 128x32 tcgen05 SYRK tile (every
    other subdomain, the rest 32x32 or FP64): the tile tasks' union lists,
    their cut rule and their epilogue, replayed in FP64 on the CPU, give the
    oracle's F with every entry written; every 16-byte copy the kernel issues
    stays inside its supernode's digit block and the stage."""
    fs = host.factorize_problem(prob.subdomains)
    n = len(fs)
    var = [(5, 7, 0)[i % 3] for i in range(n)]
    tile = [i % 2 for i in range(n)]
    plan = sc.Plan(fs, prob.n_dual, sub_slices=var, sub_tile=tile)
    tile_subs = {i for i in range(n) if tile[i] and var[i]}
    T = pe.export_plan(plan)
    pe.check_bounds(T, plan.sizes, plan.stats, tile_subs)
    lay = pe.check_split_layout(T, plan.sizes, plan.stats, sub_var=[v | (8 if i in tile_subs else 0)
                                                                  for i, v in enumerate(var)])
    for t in T["syrk"]:
        if int(t["sub"]) in tile_subs:
            pe.check_tile_fetches(T, t, lay["yd_plane"], var[int(t["sub"])])
    F = pe.emulate_assembly(T, plan.sizes, plan.stats, sc.concat_L_values(fs), tile_subs)
    assert not np.isnan(F).any(), "F entries left unwritten"
    Fo = oracle.dual_operators(prob.subdomains)
    for i in range(n):
        assert oracle.relative_frobenius(pe.export_dense(T, F, i), Fo[i]) <= 1e-12
    ntile = sum(1 for t in T["syrk"] if int(t["sub"]) in tile_subs)
    assert ntile > 0


def test_tile_options_validated():
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    with pytest.raises(sc.SCError):
        sc.Plan(fs, prob.n_dual, sub_slices=[5] * len(fs), sub_tile=[2] * len(fs))
    with pytest.raises(sc.SCError):
        sc.Plan(fs, prob.n_dual, tile=3)
    with pytest.raises(sc.SCError):
        sc.Plan(fs, prob.n_dual, poll_limit=-1)


def _dense_factor_plan_stats(n, m):
    """Plan counters for a dense lower factor (one supernode) with the
    perfectly triangular right-hand side of paper Sec. 4.3: the pivot of
    column i is row i n / m."""
    cp = np.zeros(n + 1, np.int64)
    cp[1:] = np.cumsum(n - np.arange(n))
    ri = np.concatenate([np.arange(c, n) for c in range(n)]).astype(np.int32)
    piv = ((np.arange(m) * n) // m).astype(np.int32)
    btc = np.arange(m + 1, dtype=np.int32)
    lam = np.arange(m, dtype=np.int32)
    sg = np.ones(m, np.int8)
    d = abi.SubdomainDesc()
    d.n, d.m = n, m
    d.L_colptr, d.L_rowind, d.Bt_colptr = cp.ctypes.data, ri.ctypes.data, btc.ctypes.data
    d.Bt_rowind, d.Bt_sign, d.lambda_map = piv.ctypes.data, sg.ctypes.data, lam.ctypes.data
    lib = _native.sc_lib()
    h = ctypes.c_void_p()
    assert lib.sc_plan(ctypes.byref(h), 1, ctypes.byref(d), m, None) == 0
    s = abi.Stats()
    lib.sc_get_stats(h, ctypes.byref(s))
    lib.sc_destroy(h)
    return s


def test_perfect_triangle_flop_ratio():
    """Paper Sec. 4.3: for a perfectly triangular RHS, dense TRSM and SYRK do 3x
    the flops of the pivot-pruned ones (pyramid vs prism).  The plan's own
    counters approach 3 as the 32-row blocks get small relative to n."""
    ratios = []
    for n, m in [(256, 128), (1024, 512), (2048, 1024)]:
        s = _dense_factor_plan_stats(n, m)
        assert s.n_supernodes == 1
        ratios.append(s.flops_dense / (s.flops_trsm + s.flops_syrk))
    assert ratios[0] < ratios[1] < ratios[2] < 3.0
    assert ratios[2] > 2.85


def test_perfect_triangle_emulation():
    """The cut-trimmed plan still produces F exactly on a dense factor."""
    rng = np.random.default_rng(3)
    n, m = 150, 70
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)
    G = np.linalg.cholesky(A)
    cp = np.zeros(n + 1, np.int64)
    cp[1:] = np.cumsum(n - np.arange(n))
    ri = np.concatenate([np.arange(c, n) for c in range(n)]).astype(np.int32)
    vals = np.concatenate([G[c:, c] for c in range(n)])
    piv = ((np.arange(m) * n) // m).astype(np.int32)
    sign = rng.choice([-1, 1], size=m).astype(np.int8)
    L = host.HostFactor(n, cp, ri, vals, np.arange(n, dtype=np.int32))
    fs = host.FactoredSubdomain(L, np.arange(m + 1, dtype=np.int32), piv, sign, np.arange(m, dtype=np.int32))
    plan = sc.Plan([fs], m)
    T = pe.export_plan(plan)
    pe.check_bounds(T, plan.sizes, plan.stats)
    F = pe.export_dense(T, pe.emulate_assembly(T, plan.sizes, plan.stats, vals), 0)
    Bt = np.zeros((n, m))
    Bt[piv, np.arange(m)] = sign
    ref = Bt.T @ np.linalg.solve(A, Bt)
    assert oracle.relative_frobenius(F, ref) < 1e-12


@pytest.mark.parametrize("planned", [True, False])
@pytest.mark.parametrize("threads", [1, 3])
def test_host_implicit_apply_matches_oracle(threads, planned):
    for prob in (synth.cube_heat_3d(2, 4, coef_seed=2), edge_batch(), synth.elasticity_cubes((2, 1, 1), 2, 4, seed=1)):
        fs = host.factorize_problem(prob.subdomains)
        lam = np.random.default_rng(9).standard_normal(prob.n_dual)
        q = host.ImplicitApply(fs, prob.n_dual, planned=planned)(lam, threads=threads)
        Fo = [oracle.dual_operator(sd, refine=1) if sd.m else np.zeros((0, 0)) for sd in prob.subdomains]
        qo = oracle.apply_dual(Fo, [s.lambda_map for s in prob.subdomains], lam, prob.n_dual)
        assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)


def test_host_implicit_plan_checks_patterns_entry_by_entry():
    """A lower-triangular L whose neighbouring columns have matching counts
    and parents but different rows must not be merged into one supernode: the
    planned apply equals the column-by-column one (and a dense solve) on it,
    with several nonzeros per B^T column and an empty one."""
    rng = np.random.default_rng(5)
    n = 12
    cols = {0: [0, 1, 3, 7], 1: [1, 2, 5], 2: [2, 5, 9], 3: [3, 4], 4: [4, 6], 5: [5, 9, 11], 6: [6, 7],
            7: [7, 8], 8: [8, 10], 9: [9, 11], 10: [10, 11], 11: [11]}
    colptr = np.zeros(n + 1, np.int64)
    rowind, vals = [], []
    for c in range(n):
        rows = cols[c]
        rowind += rows
        vals += [3.0 + rng.uniform()] + list(rng.uniform(-0.5, 0.5, len(rows) - 1))
        colptr[c + 1] = len(rowind)
    L = host.HostFactor(n, colptr, np.array(rowind, np.int32), np.array(vals), np.arange(n, dtype=np.int32))
    Bt = sp.csc_matrix(([1.0, -1.0, 1.0, 1.0, -1.0], ([0, 4, 8, 11, 2], [0, 0, 1, 2, 3])), shape=(n, 5))
    fsd = host.FactoredSubdomain(L=L, bt_colptr=Bt.indptr.astype(np.int32), bt_rowind=Bt.indices.astype(np.int32),
                                 bt_sign=Bt.data.astype(np.int8), lambda_map=np.array([4, 0, 2, 1, 3], np.int32))
    lam = rng.standard_normal(5)
    qp = host.ImplicitApply([fsd], 5, planned=True)(lam, threads=1)
    qc = host.ImplicitApply([fsd], 5, planned=False)(lam, threads=1)
    Ld = sp.csc_matrix((L.values, L.rowind, L.colptr), shape=(n, n)).toarray()
    Bd = Bt.toarray()
    Fd = Bd.T @ np.linalg.solve(Ld.T, np.linalg.solve(Ld, Bd))
    qd = np.zeros(5)
    np.add.at(qd, fsd.lambda_map, Fd @ lam[fsd.lambda_map])
    assert np.allclose(qp, qd, rtol=1e-13, atol=1e-13) and np.allclose(qc, qd, rtol=1e-13, atol=1e-13)


def test_mlp_header_symbols_exported():
    names = _declared("sc_mlp.h")
    lib = _native.sc_lib()
    assert names and all(hasattr(lib, n) for n in names)


def test_workspace_waves_bound_the_workspace():
    """ws_limit packs subdomains into waves that reuse one workspace."""
    prob = synth.cube_heat_3d(2, 5)
    fs = host.factorize_problem(prob.subdomains)
    one = sc.Plan(fs, prob.n_dual)
    lim = one.sizes.ws_bytes // 3
    waved = sc.Plan(fs, prob.n_dual, ws_limit=lim)
    assert waved.stats.n_waves >= 3 and waved.sizes.ws_bytes <= lim
    assert waved.stats.y_doubles == one.stats.y_doubles
    T = pe.export_plan(waved)
    pe.check_bounds(T, waved.sizes, waved.stats)
    with pytest.raises(sc.SCError) as e:
        sc.Plan(fs, prob.n_dual, ws_limit=1000)
    assert e.value.status == abi.SC_ERR_OOM


def _general_gluing():
    """B^T columns with several nonzeros, an empty column and duplicate dofs
    (a general B, paper Sec. 3) on a 3D cube."""
    import scipy.sparse as sp
    base = synth.cube_heat_3d(parts=1, k=4).subdomains[0]
    rng = np.random.default_rng(7)
    n, m = base.n, 40
    rows, cols, vals = [], [], []
    for j in range(m):
        if j == 11:
            continue                                  # empty column
        k = 3 if j % 7 == 0 else 1
        for r in rng.choice(n, size=k, replace=False):
            rows.append(r); cols.append(j); vals.append(rng.choice([-1.0, 1.0]))
    rows.append(rows[0]); cols.append(39); vals.append(1.0)   # a dof shared by two columns
    Bt = sp.csc_matrix((vals, (rows, cols)), shape=(n, m))
    sd = synth.Subdomain(K=base.K, fixed=base.fixed, Bt=Bt, lambda_map=np.arange(m), grid=base.grid,
                         ndpn=1, key=None)
    return synth.Problem("general", [sd], m, 0)


def _implicit_cases():
    yield from _cases()
    yield "chain", synth.Problem("chain", [synth.chain_1d(40, [3, 17, 40])], 3, 0)
    yield "cube_2x8", synth.cube_heat_3d(2, 8)         # 81-column top separators: three 32-column blocks


@pytest.mark.parametrize("name,prob", list(_implicit_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_implicit_plan_emulation_matches_oracle(name, prob):
    """The GPU implicit apply's plan (levels, panels, B^T gather/scatter),
    replayed on the CPU with the kernel's index formulas, gives F*lambda."""
    fs = host.factorize_problem(prob.subdomains)
    ip = implicit.ImplicitPlan(fs, prob.n_dual)
    T = ie.export_plan(ip)
    Loff = np.concatenate([[0], np.cumsum([f.L.values.size for f in fs])])
    assert ip.sizes.L_values == Loff[-1]
    ie.check_bounds(T, ip.sizes, Loff, prob.n_dual)
    lam = np.random.default_rng(5).standard_normal(prob.n_dual)
    q = ie.emulate(T, ip.sizes, sc.concat_L_values(fs), lam, prob.n_dual)
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains), [s.lambda_map for s in prob.subdomains],
                           lam, prob.n_dual)
    assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)
    # visited entries and levels are what the plan claims
    sns = T["sns"]
    nnz = sum(int(s["ns"]) * (int(s["ns"]) + 1) // 2 + int(s["ns"]) * int(s["rs"]) for s in sns)
    assert ip.sizes.nnz_visited == nnz and ip.sizes.flops == 4.0 * nnz


def test_implicit_plan_general_gluing_and_order():
    prob = _general_gluing()
    fs = host.factorize_problem(prob.subdomains)
    ip = implicit.ImplicitPlan(fs, prob.n_dual)
    T = ie.export_plan(ip)
    Loff = np.concatenate([[0], np.cumsum([f.L.values.size for f in fs])])
    ie.check_bounds(T, ip.sizes, Loff, prob.n_dual)
    lam = np.random.default_rng(2).standard_normal(prob.n_dual)
    q = ie.emulate(T, ip.sizes, sc.concat_L_values(fs), lam, prob.n_dual)
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains), [s.lambda_map for s in prob.subdomains],
                           lam, prob.n_dual)
    assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)


def test_implicit_cluster_items():
    """Automatic rule: large subdomains get a cluster each, small ones are
    packed eight to a cluster; 0 and a huge threshold select all / none."""
    prob = synth.mixed_batch(lat2d=(4, 4), k2d=(6, 40), lat3d=(2, 2, 1), k3d=(2, 6), seed=2)
    fs = host.factorize_problem(prob.subdomains)
    Loff = np.concatenate([[0], np.cumsum([f.L.values.size for f in fs])])
    nnz = implicit.ImplicitPlan(fs, prob.n_dual).sizes.nnz_visited
    for cmw, kinds in ((0, {0}), (1 << 60, {1}), (1, {0}), (nnz // 40, {0, 1})):
        ip = implicit.ImplicitPlan(fs, prob.n_dual, cluster_min_work=cmw, pairs=-1)
        T = ie.export_plan(ip)
        ie.check_bounds(T, ip.sizes, Loff, prob.n_dual)
        got = set(int(k) for k in T["items"]["kind"])
        if kinds is not None:
            assert got == kinds, (cmw, got)
        assert ip.sizes.n_cluster_subdomains == int(np.sum(T["items"]["kind"] == 0))


def test_implicit_pair_items():
    """CTA pairs (on request): every pair subdomain splits into two non-empty
    parts touching disjoint rows, with the scatter grouped by part
    (check_pair_split); the plan replayed in its level order reproduces the
    oracle; the automatic rule keeps one CTA per subdomain; invalid option
    values are refused."""
    prob = synth.mixed_batch(lat2d=(4, 4), k2d=(6, 40), lat3d=(2, 2, 1), k3d=(2, 6), seed=2)
    fs = host.factorize_problem(prob.subdomains)
    Loff = np.concatenate([[0], np.cumsum([f.L.values.size for f in fs])])
    lam = np.random.default_rng(4).standard_normal(prob.n_dual)
    Lv = np.concatenate([f.L.values for f in fs])
    qo = oracle.apply_dual(oracle.dual_operators(prob.subdomains, refine=1), [s.lambda_map for s in prob.subdomains],
                           lam, prob.n_dual)
    for pairs in (0, 1):
        ip = implicit.ImplicitPlan(fs, prob.n_dual, cluster_min_work=1 << 60, pairs=pairs)
        T = ie.export_plan(ip)
        ie.check_bounds(T, ip.sizes, Loff, prob.n_dual)
        kinds = set(int(k) for k in T["items"]["kind"])
        if pairs == 0:
            assert kinds == {1}, kinds
            continue
        assert 2 in kinds, kinds
        npair = sum(int(it["n"]) for it in T["items"] if it["kind"] == 2)
        assert npair >= len(fs) // 2
        q = ie.emulate(T, ip.sizes, Lv, lam, prob.n_dual)
        assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)
    with pytest.raises(sc.SCError, match="pairs"):
        implicit.ImplicitPlan(fs, prob.n_dual, pairs=2)


def test_implicit_plan_subdomain_order_and_validation():
    prob = synth.elasticity_cubes((2, 1, 1), 2, 4, seed=3)
    fs = host.factorize_problem(prob.subdomains)
    ip = implicit.ImplicitPlan(fs, prob.n_dual)
    T = ie.export_plan(ip)
    work = [int(np.sum(T["sns"][sd["sn_lo"]:sd["sn_hi"]]["ns"] * (T["sns"][sd["sn_lo"]:sd["sn_hi"]]["ns"] + 1) // 2
                       + T["sns"][sd["sn_lo"]:sd["sn_hi"]]["ns"] * T["sns"][sd["sn_lo"]:sd["sn_hi"]]["rs"]))
            for sd in T["subs"]]
    assert work == sorted(work, reverse=True), "subdomains are launched largest first"
    with pytest.raises(sc.SCError, match="lambda_map out of range"):
        implicit.ImplicitPlan(fs, prob.n_dual - 1 if prob.n_dual > 1 else 0)


def test_pipeline_refactorisation_reproduces_the_planned_factor():
    """The pipeline refactorises with the final ordering and no further
    reordering; that must give the very L the plans were made for."""
    prob = synth.elasticity_cubes((2, 1, 1), 2, 4, seed=1)
    fs = host.factorize_problem(prob.subdomains)
    for sd, f in zip(prob.subdomains, fs):
        g = host.factorize(sd.K, sd.fixed, perm=f.L.perm, postorder=False)
        assert np.array_equal(g.colptr, f.L.colptr) and np.array_equal(g.rowind, f.L.rowind)
        assert np.array_equal(g.values, f.L.values)


def test_pipeline_create_validates_chunks():
    """Chunks must cover every subdomain once and match their plans (checked
    before any CUDA call)."""
    lib = _native.pipe_lib()
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    nsub = len(fs)
    p0, p1 = sc.Plan(fs[:4], prob.n_dual), sc.Plan(fs[4:], prob.n_dual)
    subs = (abi.PipeSubdomain * nsub)()
    keep = []
    for i, (sd, f) in enumerate(zip(prob.subdomains, fs)):
        K = sd.K.tocsc()
        K.sort_indices()
        arrs = [np.ascontiguousarray(K.indptr, np.int64), np.ascontiguousarray(K.indices, np.int32),
                np.ascontiguousarray(K.data), np.ascontiguousarray(sd.fixed, np.int32),
                np.ascontiguousarray(f.L.perm, np.int32)]
        keep += arrs
        subs[i].n = K.shape[0]
        subs[i].K_colptr, subs[i].K_rowind, subs[i].K_val = [a.ctypes.data for a in arrs[:3]]
        subs[i].nfixed, subs[i].fixed, subs[i].perm = len(arrs[3]), arrs[3].ctypes.data, arrs[4].ctypes.data

    def run(ranges, plans):
        ch = (abi.PipeChunk * len(ranges))()
        for c, ((lo, hi), p) in enumerate(zip(ranges, plans)):
            ch[c].lo, ch[c].hi, ch[c].plan = lo, hi, p.h.value
            ch[c].L_dev = ch[c].F_dev = ch[c].ws_dev = 256       # never dereferenced: validation fails first
            ch[c].ws_bytes = 1 << 40
        h = ctypes.c_void_p()
        st = lib.scp_create(ctypes.byref(h), nsub, subs, len(ranges), ch, 2)
        msg = lib.scp_last_error(h).decode()
        lib.scp_destroy(h)
        return st, msg

    st, msg = run([(0, 4)], [p0])
    assert st == abi.SC_ERR_INVALID_ARG and "exactly one chunk" in msg
    st, msg = run([(0, 3), (3, nsub)], [p0, p1])
    assert st == abi.SC_ERR_INVALID_ARG and "hi - lo" in msg
    st, msg = run([(0, 4), (2, nsub)], [p0, p1])
    assert st == abi.SC_ERR_INVALID_ARG
    # the symbolic stage runs in scp_create: a subdomain whose ordering is not
    # the one its plan was made for has another L pattern and is refused there
    ident = np.arange(subs[2].n, dtype=np.int32)
    keep.append(ident)
    good_perm = subs[2].perm
    subs[2].perm = ident.ctypes.data
    st, msg = run([(0, 4), (4, nsub)], [p0, p1])
    subs[2].perm = good_perm
    assert st == abi.SC_ERR_INVALID_ARG and "subdomain 2" in msg and "the plan expects" in msg, msg


def test_plan_rejects_bad_persistent_flag():
    """sc_options.persistent is 0 or 1."""
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    lib = _native.sc_lib()
    keep = []
    d = _desc_from(fs[0], keep)
    for flag, ok in ((0, True), (1, True), (2, False)):
        opt = abi.Options()
        opt.persistent = flag
        h = ctypes.c_void_p()
        st = lib.sc_plan(ctypes.byref(h), 1, ctypes.byref(d), prob.n_dual, ctypes.byref(opt))
        msg = lib.sc_last_error(h).decode() if h.value else ""
        if h.value:
            lib.sc_destroy(h)
        assert (st == abi.SC_OK) == ok, (flag, st, msg)
        if not ok:
            assert "persistent" in msg


def test_pack_is_the_inverse_of_export():
    """Plan.pack writes dense symmetric m_i x m_i matrices into the plan's F
    layout: tile (I, J), J <= I, at I (I + 1) / 2 + J, entry (r, c) of a tile
    at r + 32 c, diagonal tiles full, padding zero; the plan replay's export
    reads them back unchanged."""
    torch = pytest.importorskip("torch")
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual)
    assert any(m % 32 for m in plan.m) and max(plan.m) > 32
    rng = np.random.default_rng(11)
    mats = []
    for m in plan.m:
        A = rng.standard_normal((m, m))
        mats.append(A + A.T)
    buf = plan.pack(mats, device="cpu").numpy()
    assert buf.shape == (max(1, plan.sizes.F_doubles),)
    T = pe.export_plan(plan)
    for i, M in enumerate(mats):
        m = plan.m[i]
        nt = (m + 31) // 32
        off = int(plan.F_offsets[i])
        for I in range(nt):
            for J in range(I + 1):
                tile = buf[off + (I * (I + 1) // 2 + J) * 1024:][:1024].reshape(32, 32)   # [c, r]
                want = np.zeros((32, 32))
                rows, cols = min(32, m - 32 * I), min(32, m - 32 * J)
                want[:cols, :rows] = M[32 * I:32 * I + rows, 32 * J:32 * J + cols].T
                assert np.array_equal(tile, want)
        assert np.array_equal(pe.export_dense(T, buf, i), M)


@pytest.mark.parametrize("name,prob", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_plan_predicts_the_structure_of_Y(name, prob):
    """Structural pins on Y = L^{-1} P B^T (paper Sec. 3.2): computed here
    with a plain sparse triangular solve (scipy), independent of the plan,
    every nonzero of Y lies where the plan keeps Y (rows of a supernode s,
    sorted columns [jlo_s, jhi_s), and within the column cut of the row's
    32-row block); Y(r, j) = 0 above the pivot p_j (sorted columns, so the
    pruning by pivots is never lossy); and the pivots are non-decreasing in
    the sorted order."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual)
    T = pe.export_plan(plan)
    sns = T["sns"]
    kept_total = nnz_total = 0
    for i, f in enumerate(fs):
        sd = T["subs"][i]
        n, m = f.n, f.m
        if m == 0:
            continue
        L = sp.csc_matrix((f.L.values, f.L.rowind, f.L.colptr), shape=(n, n))
        Bt = sp.csc_matrix((f.bt_sign.astype(float), f.bt_rowind, f.bt_colptr), shape=(n, m))
        perm = T["perm"][sd["col_off"]:sd["col_off"] + m]
        Bs = Bt[:, perm]
        piv = np.array([Bs.indices[Bs.indptr[j]:Bs.indptr[j + 1]].min() for j in range(m)])
        assert np.all(np.diff(piv) >= 0)
        Y = spla.spsolve_triangular(L.tocsr(), Bs.toarray(), lower=True)
        nz = Y != 0.0
        assert not np.any(nz & (np.arange(n)[:, None] < piv[None, :])), "Y nonzero above a pivot"
        kept = np.zeros((n, m), bool)
        for s in sns[sns["sub"] == i]:
            for kb in range(0, s["ns"], 32):
                cut = min(int(s["jhi"]), int(T["cuts"][s["cut_off"] + kb // 32]))
                r0 = s["c0"] + kb
                kept[r0:r0 + min(32, s["ns"] - kb), s["jlo"]:cut] = True
        assert not np.any(nz & ~kept), f"subdomain {i}: Y nonzero where the plan keeps none"
        kept_total += kept.sum()
        nnz_total += nz.sum()
    assert nnz_total > 0 and kept_total >= nnz_total


@pytest.mark.parametrize("case", ["L_row_out_of_range", "L_diag_not_first", "L_rows_unsorted", "L_colptr_start",
                                  "Bt_colptr_decreasing", "Bt_row_out_of_range", "lambda_out_of_range"])
def test_host_implicit_apply_rejects_bad_patterns(case):
    """Both host implicit entry points check every index the solves form
    (scf_implicit_apply on each call, scf_implicit_plan once)."""
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    f = fs[2]
    L = host.HostFactor(f.L.n, f.L.colptr.copy(), f.L.rowind.copy(), f.L.values, f.L.perm)
    btc, btr, lam = f.bt_colptr.copy(), f.bt_rowind.copy(), f.lambda_map.copy()
    c = 7
    a = int(L.colptr[c])
    if case == "L_row_out_of_range":
        L.rowind[int(L.colptr[c + 1]) - 1] = f.n
    elif case == "L_diag_not_first":
        L.rowind[a], L.rowind[a + 1] = L.rowind[a + 1], L.rowind[a]
    elif case == "L_rows_unsorted":
        L.rowind[a + 1], L.rowind[a + 2] = L.rowind[a + 2], L.rowind[a + 1]
    elif case == "L_colptr_start":
        L.colptr[0] = 1
    elif case == "Bt_colptr_decreasing":
        btc[3] = btc[5]
    elif case == "Bt_row_out_of_range":
        btr[4] = f.n
    else:
        lam[0] = prob.n_dual
    bad = host.FactoredSubdomain(L=L, bt_colptr=btc, bt_rowind=btr, bt_sign=f.bt_sign, lambda_map=lam)
    subs = fs[:2] + [bad] + fs[3:]
    x = np.ones(prob.n_dual)
    with pytest.raises(RuntimeError):
        host.ImplicitApply(subs, prob.n_dual, planned=False)(x)
    with pytest.raises(RuntimeError):
        host.ImplicitApply(subs, prob.n_dual, planned=True)


def test_add_symmetric_batch_matches_pack():
    """Plan.add_symmetric_batch scatters lower-triangle entries (r >= c, with
    repeats, which accumulate) of several subdomains into F's layout: on a
    zero buffer it gives exactly the pack of the symmetric matrices they
    define (an off-diagonal-tile pair stored once, a diagonal tile both
    entries); the one-subdomain form agrees."""
    torch = pytest.importorskip("torch")
    prob = synth.cube_heat_3d(2, 3)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual)
    rng = np.random.default_rng(12)
    entries, mats = [], []
    for i, m in enumerate(plan.m):
        n = 4 * m
        r, c = rng.integers(0, m, n), rng.integers(0, m, n)
        r, c = np.maximum(r, c), np.minimum(r, c)
        v = rng.integers(-8, 8, n).astype(np.float64)    # small integers: sums exact in any order
        A = np.zeros((m, m))
        np.add.at(A, (r, c), v)
        mats.append(A + np.tril(A, -1).T)
        entries.append((i, r, c, v))
    want = plan.pack(mats, device="cpu")
    got = torch.zeros_like(want)
    plan.add_symmetric_batch(got, entries)
    assert torch.equal(got, want)
    one = torch.zeros_like(want)
    for e in entries:
        plan.add_symmetric(one, *e)
    assert torch.equal(one, want)


def test_trsm_tasks_in_snake_order_of_largest_first():
    """The planner hands the FP64 TRSM tasks out largest first by its cost
    estimate (32 lanes x (kw^2 + 2 kw rows below) per nonempty 32-row block,
    plus 1e3 per supernode in the list), with every other round of 152 tasks
    reversed (one round per SM of a GB300): undoing the reversals gives a
    non-increasing cost sequence, and the odd rounds run smallest first."""
    prob = synth.make_config(2)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual)
    T = pe.export_plan(plan)
    pe.check_bounds(T, plan.sizes, plan.stats)
    sns, cuts = T["sns"], T["cuts"]
    cost = []
    for t in T["trsm"]:
        lst = T["trsm_list"][t["list_off"]:t["list_off"] + t["list_len"]]
        c_lo, c_hi = int(t["c_lo"]), int(t["c_lo"]) + int(t["w"])
        exe = 0
        for si in lst:
            s = sns[si]
            a, b = max(int(s["jlo"]), c_lo), min(int(s["jhi"]), c_hi)
            ns, nrow = int(s["ns"]), int(s["ns"]) + int(s["rs"])
            for kb in range(0, ns, 32):
                if min(b, int(cuts[int(s["cut_off"]) + kb // 32])) - a <= 0:
                    continue
                kw = min(32, ns - kb)
                exe += 32 * (kw * kw + 2 * kw * (nrow - kb - kw))
        cost.append(exe + 1000 * int(t["list_len"]))
    assert len(cost) > 4 * 152
    rounds = [cost[r:r + 152] for r in range(0, len(cost), 152)]
    unsnaked = [c for k, r in enumerate(rounds) for c in (r[::-1] if k % 2 else r)]
    assert all(x >= y for x, y in zip(unsnaked, unsnaked[1:]))
    assert any(r[0] < r[-1] for r in rounds[1::2])
