"""Per-subdomain kernel-variant selection: measuring autotuner and learned predictor.

The assembly offers, per subdomain, FP64 or split precision with 3..7 digits
(include/sc.h, sc_options.sub_slices) and, for split precision, two SYRK
output tiles: 32x32 blocks on the warp-level tensor-core instruction or
128x32 tiles on tcgen05 (sc_options.sub_tile).  Which one is fastest depends
on the subdomain (small or narrow subdomains do not repay the digit-plane
overhead or fill the large tile; large ones gain up to ~3x), and which ones
are accurate enough depends on the error target.  This module

  * describes every subdomain by sparsity-pattern features from its plan
    (sizes, supernode structure, flop counts) and one value feature (the
    spread of L's diagonal, a conditioning proxy);
  * ``autotune``: measures, for every structural class of subdomains, the
    per-subdomain time of each variant (replicated sub-batches timed with
    CUDA events) and its error against the FP64 variant;
  * ``LearnedSelector``: trains the GPU MLP (include/sc_mlp.h) on those
    records to predict log time and log error of every variant from the
    features, and picks per subdomain the fastest variant predicted to meet
    the error target -- through the C ABI (sc_select: the library computes the
    features from the plan, runs the forward pass and applies the rule).
    Classes the autotuner has measured keep its measured
    choice (the fallback); on the others the measured choice, when available,
    is the yardstick of the learned choice's regret.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import abi, sc

# A variant is coded as digits + 8 * tile: 0 = FP64; S = split with S digits and
# 32x32 SYRK blocks (mma.sync); 8 + S = S digits with the 128x32 SYRK tile on
# tcgen05 (include/sc.h: sub_slices, sub_tile).  The structural choice (tile)
# and the arithmetic one (digits) are chosen jointly.
TILE = 8
VARIANTS: Tuple[int, ...] = (0, 7, 7 + TILE, 5, 5 + TILE)


def digits(v: int) -> int:
    return int(v) & 7


def tile(v: int) -> int:
    return int(v) >> 3


def plan_options(var: Sequence[int]) -> dict:
    """sc.Plan keyword arguments for per-subdomain variant codes."""
    return {"sub_slices": [digits(v) for v in var], "sub_tile": [tile(v) for v in var]}
FEATURES = ("log2_n", "log2_m", "log2_nnzL", "log2_supernodes", "log2_max_supernode", "log2_flops_trsm",
            "log2_flops_syrk", "log2_flops_dense", "log2_y_doubles", "log2_diag_spread")


def _log2(x: float) -> float:
    return math.log2(max(float(x), 1.0))


def class_key(f) -> tuple:
    """Structural class: the same factor pattern (n, nnz(L) and its row
    indices) and a multiplier count in the same quarter-octave; the finer
    differences (which dofs are glued) are left to the learned features."""
    return (f.n, f.L.nnz, int(round(4 * math.log2(max(f.m, 1)))), hash(f.L.rowind.tobytes()))


def subdomain_features(fs: Sequence, plan=None) -> np.ndarray:
    """[nsub, len(FEATURES)], computed by the library from the batch plan
    (include/sc.h, sc_subdomain_features), the same features sc_select uses."""
    import ctypes
    if plan is None:
        plan = sc.Plan(fs, max((int(np.max(f.lambda_map)) + 1 for f in fs if f.m), default=1))
    out = np.zeros((len(fs), abi.SC_NUM_FEATURES), np.float32)
    vals = sc.concat_L_values(fs)
    rc = plan.lib.sc_subdomain_features(plan.h, vals.ctypes.data if vals.size else None,
                                        out.ctypes.data if out.size else None)
    if rc != 0:
        raise sc.SCError(rc, plan.lib.sc_last_error(plan.h).decode())
    return out.astype(np.float64)


@dataclasses.dataclass
class ClassRecord:
    key: tuple
    members: List[int]
    features: np.ndarray                 # of the representative
    time_ms: Dict[int, float]            # per subdomain, per variant
    error: Dict[int, float]              # relative Frobenius vs the FP64 variant


def _time_variant(batch, n_dual, v, device, reps):
    import torch
    plan = sc.Plan(batch, n_dual, **plan_options([v] * len(batch))).upload(device)
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
    """Measure every (or the listed) structural class of the batch, over the
    joint (digits, SYRK tile) variant space."""
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
        """Variant codes for feature rows X (the rule of sc_select, evaluated here)."""
        times, errs = self.predict(X)
        return [best_variant(t, e, tol, margin) for t, e in zip(times, errs)]

    def c_selector(self):
        """The trained network as an include/sc.h sc_selector (kept alive on self)."""
        import ctypes
        self._sel_arrays = [np.ascontiguousarray(a) for a in (
            np.array([digits(v) for v in self.variants], np.int8), np.array([tile(v) for v in self.variants], np.int8),
            self.net.mu.astype(np.float32), self.net.sd.astype(np.float32),
            self.tmu.astype(np.float32), self.tsd.astype(np.float32))]
        sl, tl, xm, xs, ym, ys = self._sel_arrays
        return abi.Selector(len(self.variants), sl.ctypes.data, tl.ctypes.data, self.net.dims[1],
                            self.net.params.data_ptr(), xm.ctypes.data, xs.ctypes.data, ym.ctypes.data, ys.ctypes.data)

    def select_batch(self, fs: Sequence, tol: float, margin: float = 10.0, plan=None) -> List[int]:
        """Per-subdomain variant codes through the C ABI (sc_select): the
        library computes the features from the plan, runs the network's
        forward pass on the GPU and applies the choice rule."""
        import ctypes

        import torch
        if plan is None:
            plan = sc.Plan(fs, max((int(np.max(f.lambda_map)) + 1 for f in fs if f.m), default=1))
        sel = self.c_selector()
        need = ctypes.c_size_t()
        plan._check(plan.lib.sc_select_workspace(plan.h, ctypes.byref(sel), ctypes.byref(need)))
        ws = torch.empty(max(1, need.value), dtype=torch.float32, device=self.net.device)
        vals = sc.concat_L_values(fs)
        sl = np.zeros(len(fs), np.int8)
        tl = np.zeros(len(fs), np.int8)
        plan._check(plan.lib.sc_select(plan.h, ctypes.byref(sel), vals.ctypes.data if vals.size else None,
                                       float(tol), float(margin), ws.data_ptr(), ws.numel(),
                                       sl.ctypes.data, tl.ctypes.data, None))
        return [int(s) + TILE * int(t) for s, t in zip(sl, tl)]


def select(fs: Sequence, tol: float, selector: Optional[LearnedSelector] = None,
           measured: Optional[Dict[tuple, ClassRecord]] = None, margin: float = 10.0) -> List[int]:
    """Per-subdomain variant codes: measured classes use the autotuner's
    choice, the others the learned prediction through sc_select (FP64 when
    neither is available)."""
    out = [0] * len(fs)
    if selector is not None:
        out = selector.select_batch(fs, tol, margin)
    for i, f in enumerate(fs):
        rec = measured.get(class_key(f)) if measured else None
        if rec is not None:
            out[i] = best_variant(rec.time_ms, rec.error, tol)
    return out
