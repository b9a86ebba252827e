"""Full-size parity: every subdomain of configs 3, 4 and 5, through the C ABI,
against the memoised, refined FP64 oracle (tests/fullsize.py).

  * config 3 -- 512 elasticity cubes (k 8..16), FP64 path;
  * config 4 -- config 2 (64 x 4913 dofs) in split precision, 7 and 5 digits;
  * config 5 -- 1024 2D heat squares + 1024 elasticity cubes, FP64 path, and
                the learned per-subdomain variant mix over digits x SYRK tile
                (autotuner + GPU-trained MLP + sc_select, the pipeline the
                benchmark runs).

Bounds: the FP64 path and 7 digits, 1e-12 per subdomain, or -- where an exact
solve with the library's own FP64 factor already misses the oracle (the FP64
input floor at kappa(K_reg) ~ 1e6) -- 1e-12 above that floor and 1e-12
against that exact solve.  5 digits (config 4): 2^-40 x 2e3 ~ 1.8e-9, the
digit truncation 2^-8S with the growth factor the small-case split test uses
(1e3) doubled for config 2's larger multiplier counts (m up to 1634, about
twice the square root of the small cases' m).  The learned mix: every
subdomain within the error target the selection was asked to meet (1e-8) and
FP64 / 7-digit subdomains within the FP64 bound.

Every subdomain is compared.  Where a distinct matrix's glued dofs are too
many for the oracle's flop budget, its subdomains are compared on the
complete F columns of a seeded sample of those dofs (reported).
"""
import numpy as np
import pytest

import oracle
import synth
from fullsize import TOL, FullCheck
from paper_2509_21037_gb300 import abi, host, sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# flops of oracle substitution per distinct matrix before its glued dofs are sampled
BUDGET = 1.5e12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _assemble(fs, n_dual, dev, Lv, **kw):
    plan = sc.Plan(fs, n_dual, **kw).upload(dev)
    F = plan.new_F(dev)
    F.fill_(float("nan"))                # every entry must be written by the library
    plan.assemble(Lv, F)
    assert plan.device_status() == abi.SC_OK
    assert bool(torch.isfinite(F).all()), "unwritten (NaN) entries in the F buffer"
    return plan, F


def _report(name, errs, ncols, fs, fc):
    m = np.array([f.m for f in fs])
    print(f"{name}: {len(errs)} subdomains compared, {ncols.sum()} of {m.sum()} columns "
          f"({100 * ncols.sum() / max(m.sum(), 1):.1f} %), max rel. Frobenius error {errs.max():.3e}, "
          f"median {np.median(errs):.3e}; oracle {fc.oracle_s:.1f} s")
    fl = getattr(fc, "floor_cases", [])
    if fl:
        print(f"  {len(fl)} subdomains above 1e-12 against the oracle, all at the FP64 input floor: "
              f"max error {max(c[1] for c in fl):.3e}, max floor {max(c[2] for c in fl):.3e}, "
              f"max error against the exact solve with their own factor {max(c[3] for c in fl):.3e}")


def test_config3_every_subdomain(dev):
    prob = synth.make_config(3)
    fs = host.factorize_problem(prob.subdomains, threads=0)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    plan, F = _assemble(fs, prob.n_dual, dev, Lv)
    fc = FullCheck(prob.subdomains, budget_flops=BUDGET)
    errs, ncols, bad = fc.compare(plan, F, dev, fs=fs)
    _report("config 3 FP64", errs, ncols, fs, fc)
    assert (ncols > 0).all(), "a subdomain was not compared"
    assert not bad, f"{len(bad)} subdomains out of bounds, first: {bad[:3]}"


def test_config4_every_subdomain_split(dev):
    prob = synth.make_config(4)
    fs = host.factorize_problem(prob.subdomains)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    fc = FullCheck(prob.subdomains, budget_flops=1e14)      # one distinct matrix: every column
    assert fc.fraction == 1.0
    for S, bound in ((7, TOL), (5, 2.0 ** -40 * 2e3)):
        plan, F = _assemble(fs, prob.n_dual, dev, Lv, precision=abi.SC_SPLIT_BF16, n_slices=S)
        errs, ncols, bad = fc.compare(plan, F, dev, fs=fs, variant_bound=lambda i: bound)
        _report(f"config 4, {S} digits", errs, ncols, fs, fc)
        assert (ncols == np.array([f.m for f in fs])).all()
        assert not bad, f"{S} digits: {len(bad)} subdomains out of bounds, first: {bad[:3]}"
        if S == 5:
            assert errs.min() > 1e-13          # really ran in reduced precision
        del plan, F


@pytest.fixture(scope="module")
def config5(dev):
    prob = synth.make_config(5)
    fs = host.factorize_problem(prob.subdomains, threads=0)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    fc = FullCheck(prob.subdomains, budget_flops=BUDGET)
    return prob, fs, Lv, fc


def test_config5_every_subdomain_fp64(dev, config5):
    prob, fs, Lv, fc = config5
    plan, F = _assemble(fs, prob.n_dual, dev, Lv, ws_limit=int(48e9))
    errs, ncols, bad = fc.compare(plan, F, dev, fs=fs)
    _report("config 5 FP64", errs, ncols, fs, fc)
    assert (ncols > 0).all(), "a subdomain was not compared"
    assert not bad, f"{len(bad)} subdomains out of bounds, first: {bad[:3]}"


def test_config5_learned_variant_mix(dev, config5):
    """The learned selection of the benchmark (autotuner on a subset of the
    structural classes, MLP trained on its records by the library's kernels,
    measured choice kept where measured), error target 1e-8, assembled in one
    batch; each subdomain against the bound of the variant it was given."""
    from paper_2509_21037_gb300 import tune
    prob, fs, Lv, fc = config5
    tol = 1e-8
    V = tune.VARIANTS
    keys = sorted({tune.class_key(f) for f in fs}, key=lambda k: (k[0], k[2], k[1]))
    recs = tune.autotune(fs, dev, variants=V, classes=keys[::9], reps=1)
    sel = tune.LearnedSelector(variants=V, device=dev)
    sel.fit(list(recs.values()), epochs=1500)
    var = np.array(tune.select(fs, tol, sel, measured=recs))
    counts = {int(v): int((var == v).sum()) for v in V}
    print(f"config 5 learned mix (target {tol:g}): {counts}, {len(recs)} classes measured of {len(keys)}")
    assert sum(counts[v] for v in V if tune.digits(v) == 5) > 0 and counts[0] > 0     # a real mix
    plan, F = _assemble(fs, prob.n_dual, dev, Lv, ws_limit=int(48e9), **tune.plan_options(var.tolist()))
    errs, ncols, bad = fc.compare(plan, F, dev, fs=fs,
                                  variant_bound=lambda i: tol if tune.digits(var[i]) == 5 else TOL)
    _report("config 5 learned mix", errs, ncols, fs, fc)
    for v in V:
        if counts[v]:
            print(f"  variant {v}: max error {errs[var == v].max():.3e}")
    assert (ncols > 0).all()
    assert not bad, f"{len(bad)} subdomains out of bounds, first: {bad[:3]}"
