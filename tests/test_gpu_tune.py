"""Autotuner and learned variant selector on a mixed 2D heat / 3D elasticity
batch, over the joint variant space (digits x SYRK tile: FP64, 7 or 5 digits
with 32x32 mma.sync blocks or 128x32 tcgen05 tiles): the MLP, trained on the
autotuner's records of half of the subdomain classes, picks variants for the
other half; the autotuner's own measurements there measure its regret; the
batch selection runs through the C ABI (sc_select) and must beat the
FP64-only batch and every uniform choice, and meet the error target."""
import numpy as np
import pytest

import synth
from paper_2509_21037_gb300 import host, sc, tune

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _batch_ms(fs, n_dual, dev, var, reps=3):
    plan = sc.Plan(fs, n_dual, **tune.plan_options(var)).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F = plan.new_F(dev)
    plan.assemble(Lv, F)
    assert plan.device_status() == 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.assemble(Lv, F)
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def test_learned_selector_gain_and_regret(dev):
    prob = synth.mixed_batch(lat2d=(6, 6), k2d=(12, 48), lat3d=(4, 3, 2), k3d=(3, 9), seed=3)
    fs = host.factorize_problem(prob.subdomains)
    V = tune.VARIANTS
    recs = tune.autotune(fs, dev, variants=V, reps=2)
    for k in sorted(recs, key=lambda k: recs[k].features[0]):
        r = recs[k]
        print(f"n={k[0]:6d} m~2^{k[2] / 4:.2f} " + " ".join(f"v{v}:{r.time_ms[v] * 1e3:8.1f}us/{r.error[v]:.0e}" for v in V))
    keys = sorted(recs, key=lambda k: (recs[k].features[0], recs[k].features[1], k[:3]))
    train, held = keys[::2], keys[1::2]
    sel = tune.LearnedSelector(variants=V, device=dev, seed=0)
    hist = sel.fit([recs[k] for k in train], epochs=3000)
    assert hist[-1] < 0.2 * hist[0]
    tol = 1e-8
    regrets, feasible = [], []
    for k in held:
        ch = sel.choose(recs[k].features[None], tol)[0]
        best = tune.best_variant(recs[k].time_ms, recs[k].error, tol)
        regrets.append(recs[k].time_ms[ch] / recs[k].time_ms[best] - 1.0)
        feasible.append(ch == 0 or recs[k].error[ch] <= tol)
    print(f"held-out classes {len(held)}: mean regret {np.mean(regrets):.3f}, max {np.max(regrets):.3f}, "
          f"feasible {np.mean(feasible):.2f}")
    assert all(feasible)
    assert np.mean(regrets) < 0.25
    # the batch choice through the C ABI: held-out classes from sc_select, measured ones from the autotuner
    var = tune.select(fs, tol, sel, measured={k: recs[k] for k in train})
    assert set(var) <= set(V)
    for i, f in enumerate(fs):
        r = recs.get(tune.class_key(f))
        if r is not None and var[i]:
            assert r.error[var[i]] <= tol, (i, var[i], r.error[var[i]])
    t_sel = _batch_ms(fs, prob.n_dual, dev, var)
    uniform = {v: _batch_ms(fs, prob.n_dual, dev, [v] * len(fs)) for v in V}
    print(f"batch ms: selected {t_sel:.2f}; uniform " + ", ".join(f"v{v} {t:.2f}" for v, t in uniform.items()) +
          f"; variants {dict(zip(*np.unique(var, return_counts=True)))}")
    assert t_sel < uniform[0]
    assert t_sel <= 1.05 * min(uniform.values())     # no worse than the best uniform (digits, tile) choice
    assert len(set(tune.tile(v) for v in var if v)) == 2 or len(set(var)) >= 2   # a real mix
