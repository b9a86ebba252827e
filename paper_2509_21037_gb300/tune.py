"""Per-subdomain kernel-variant selection: measuring autotuner and learned predictor.

The assembly offers, per subdomain, FP64 or split precision with 4..7 digits
(include/sc.h, sc_options.sub_slices).  Which one is fastest depends on the
subdomain (small or narrow subdomains do not repay the digit-plane overhead;
large ones gain up to ~3x), and which ones are accurate enough depends on the
error target.  This module

  * describes every subdomain by sparsity-pattern features from its plan
    (sizes, supernode structure, flop counts) and one value feature (the
    spread of L's diagonal, a conditioning proxy);
  * ``autotune``: measures, for every structural class of subdomains, the
    per-subdomain time of each variant (replicated sub-batches timed with
    CUDA events) and its error against the FP64 variant;
  * ``LearnedSelector``: trains the GPU MLP (include/sc_mlp.h) on those
    records to predict log time and log error of every variant from the
    features, and picks per subdomain the fastest variant predicted to meet
    the error target.  Classes the autotuner has measured keep its measured
    choice (the fallback); on the others the measured choice, when available,
    is the yardstick of the learned choice's regret.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import abi, sc

VARIANTS: Tuple[int, ...] = (0, 7, 6, 5, 4)        # 0 = FP64, k = split with k digits
FEATURES = ("log2_n", "log2_m", "log2_nnzL", "log2_supernodes", "log2_max_supernode", "log2_flops_trsm",
            "log2_flops_syrk", "log2_flops_dense", "log2_y_doubles", "log2_diag_spread")


def _log2(x: float) -> float:
    return math.log2(max(float(x), 1.0))


def class_key(f) -> tuple:
    """Structural class: the same factor pattern (n, nnz(L) and its row
    indices) and a multiplier count in the same quarter-octave; the finer
    differences (which dofs are glued) are left to the learned features."""
    return (f.n, f.L.nnz, int(round(4 * math.log2(max(f.m, 1)))), hash(f.L.rowind.tobytes()))


def subdomain_features(fs: Sequence) -> np.ndarray:
    """[nsub, len(FEATURES)]; one single-subdomain plan per structural class."""
    cache: Dict[tuple, np.ndarray] = {}
    out = np.zeros((len(fs), len(FEATURES)))
    for i, f in enumerate(fs):
        k = class_key(f)
        if k not in cache:
            p = sc.Plan([f], int(np.max(f.lambda_map)) + 1 if f.m else 1)
            st = p.stats
            cache[k] = np.array([_log2(f.n), _log2(f.m), _log2(f.L.nnz), _log2(st.n_supernodes),
                                 _log2(st.max_supernode), _log2(st.flops_trsm), _log2(st.flops_syrk),
                                 _log2(st.flops_dense), _log2(st.y_doubles), 0.0])
        v = cache[k].copy()
        d = f.L.values[f.L.colptr[:-1]]
        v[-1] = math.log2(float(d.max() / d.min()))
        out[i] = v
    return out


@dataclasses.dataclass
class ClassRecord:
    key: tuple
    members: List[int]
    features: np.ndarray                 # of the representative
    time_ms: Dict[int, float]            # per subdomain, per variant
    error: Dict[int, float]              # relative Frobenius vs the FP64 variant


def _time_variant(batch, n_dual, v, device, reps):
    import torch
    plan = sc.Plan(batch, n_dual, sub_slices=[v] * len(batch)).upload(device)
    Lv = torch.from_numpy(sc.concat_L_values(batch)).to(device)
    F = plan.new_F(device)
    plan.assemble(Lv, F)
    if plan.device_status() != 0:
        raise RuntimeError("device status not OK while tuning")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.assemble(Lv, F)
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps / len(batch), plan.export(F, 0).cpu().numpy()


def measure_class(f, device, variants=VARIANTS, reps: int = 3, target_flops: float = 1e11,
                  max_replicas: int = 512) -> Tuple[Dict[int, float], Dict[int, float]]:
    """Marginal per-subdomain time and error of each variant for one
    representative: t(R replicas) - t(R/2 replicas), per added subdomain, so
    that the fixed launch costs (shared by a whole batch) drop out; R is
    large enough that the R/2 batch already fills the GPU."""
    p = sc.Plan([f], int(np.max(f.lambda_map)) + 1 if f.m else 1)
    per = max(p.stats.flops_trsm + p.stats.flops_syrk, 1.0)
    R = int(min(max_replicas, max(16, math.ceil(target_flops / per))))
    R -= R % 2
    n_dual = int(np.max(f.lambda_map)) + 1 if f.m else 1
    times, errs, ref = {}, {}, None
    for v in variants:
        t_full, F0 = _time_variant([f] * R, n_dual, v, device, reps)
        t_half, _ = _time_variant([f] * (R // 2), n_dual, v, device, reps)
        times[v] = max((t_full * R - t_half * (R // 2)) / (R // 2), 1e-6)
        if v == 0:
            ref = F0
        errs[v] = float(np.linalg.norm(F0 - ref) / max(np.linalg.norm(ref), 1e-300)) if ref is not None else 0.0
    return times, errs


def autotune(fs: Sequence, device, variants=VARIANTS, classes: Optional[Sequence[tuple]] = None,
             reps: int = 3) -> Dict[tuple, ClassRecord]:
    """Measure every (or the listed) structural class of the batch."""
    feats = subdomain_features(fs)
    groups: Dict[tuple, List[int]] = {}
    for i, f in enumerate(fs):
        groups.setdefault(class_key(f), []).append(i)
    out = {}
    for k, mem in groups.items():
        if classes is not None and k not in classes:
            continue
        rep = mem[len(mem) // 2]                      # a middle member represents the class
        t, e = measure_class(fs[rep], device, variants, reps)
        out[k] = ClassRecord(k, mem, feats[rep], t, e)
    return out


def best_variant(time_ms: Dict[int, float], error: Dict[int, float], tol: float, margin: float = 1.0) -> int:
    """Fastest variant whose error (times margin) meets tol; FP64 always qualifies."""
    ok = [v for v in time_ms if v == 0 or error.get(v, np.inf) * margin <= tol]
    return min(ok, key=lambda v: time_ms[v])


class LearnedSelector:
    """MLP on subdomain features -> log10 time of every variant and log10
    error of every split variant; trained on autotuner records."""

    def __init__(self, variants=VARIANTS, hidden: int = 64, device="cuda", seed: int = 0):
        from .mlp import MLP
        self.variants = tuple(variants)
        self.split = tuple(v for v in self.variants if v)
        self.net = MLP(len(FEATURES), hidden, len(self.variants) + len(self.split), device=device, seed=seed)

    def _targets(self, recs: Sequence[ClassRecord]):
        T = np.zeros((len(recs), len(self.variants) + len(self.split)))
        M = np.ones_like(T)
        for r, rec in enumerate(recs):
            for j, v in enumerate(self.variants):
                T[r, j] = math.log10(rec.time_ms[v])
            for j, v in enumerate(self.split):
                e = rec.error.get(v, 0.0)
                T[r, len(self.variants) + j] = math.log10(max(e, 1e-17))
        return T, M

    def fit(self, recs: Sequence[ClassRecord], epochs: int = 3000, lr: float = 3e-3):
        X = np.stack([r.features for r in recs])
        T, M = self._targets(recs)
        self.tmu, self.tsd = T.mean(0), T.std(0) + 1e-6
        return self.net.fit(X, (T - self.tmu) / self.tsd, M, epochs=epochs, lr=lr)

    def predict(self, X: np.ndarray):
        Y = self.net.predict(X) * self.tsd + self.tmu
        nv = len(self.variants)
        times = [{v: 10 ** Y[i, j] for j, v in enumerate(self.variants)} for i in range(len(X))]
        errs = [{v: 10 ** Y[i, nv + j] for j, v in enumerate(self.split)} for i in range(len(X))]
        return times, errs

    def choose(self, X: np.ndarray, tol: float, margin: float = 10.0) -> List[int]:
        times, errs = self.predict(X)
        return [best_variant(t, e, tol, margin) for t, e in zip(times, errs)]


def select(fs: Sequence, tol: float, selector: Optional[LearnedSelector] = None,
           measured: Optional[Dict[tuple, ClassRecord]] = None, margin: float = 10.0) -> List[int]:
    """Per-subdomain variants: measured classes use the autotuner's choice,
    the others the learned prediction (FP64 when neither is available)."""
    out = [0] * len(fs)
    need = []
    for i, f in enumerate(fs):
        rec = measured.get(class_key(f)) if measured else None
        if rec is not None:
            out[i] = best_variant(rec.time_ms, rec.error, tol)
        else:
            need.append(i)
    if need and selector is not None:
        X = subdomain_features([fs[i] for i in need])
        for i, v in zip(need, selector.choose(X, tol, margin)):
            out[i] = v
    return out
