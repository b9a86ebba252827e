"""CPU emulation of the GPU kernels' index arithmetic over an exported plan.

Test infrastructure for the library (not the oracle): it parses the plan blob
(sc_export_plan), checks that every address the kernels form stays inside its
buffer, and replays the kernels' FP64 arithmetic task by task with numpy so
that the plan's logic can be compared with the oracle without a GPU.
"""
from __future__ import annotations

import ctypes

import numpy as np

SUB = np.dtype([("F_off", "<i8"), ("L_off", "<i8"), ("n", "<i4"), ("m", "<i4"), ("nt", "<i4"),
                ("col_off", "<i4"), ("lcp_off", "<i4"), ("pad", "<i4")])
SN = np.dtype([("y_off", "<i8"), ("rmap_off", "<i8"), ("ld_off", "<i8"), ("yd_off", "<i8"), ("sub", "<i4"), ("c0", "<i4"), ("ns", "<i4"),
               ("rs", "<i4"), ("jlo", "<i4"), ("jhi", "<i4"), ("lcp_off", "<i4"), ("cut_off", "<i4")])
TRSM = np.dtype([("sub", "<i4"), ("c_lo", "<i4"), ("w", "<i4"), ("list_off", "<i4"), ("list_len", "<i4"),
                 ("seed_lo", "<i4"), ("seed_hi", "<i4"), ("pad", "<i4")])
SYRK = np.dtype([("sub", "<i4"), ("q1", "<i4"), ("q2", "<i4"), ("list_off", "<i4"), ("list_len", "<i4"),
                 ("pad", "<i4", 3)])
SEED = np.dtype([("y_off", "<i8"), ("value", "<f8")])
APPLY = np.dtype([("sub", "<i4"), ("I", "<i4")])
HEADER = np.dtype([("magic", "<u4"), ("version", "<u4"), ("nsub", "<i4"), ("chunk", "<i4"),
                   ("n_sns", "<i8"), ("n_trsm", "<i8"), ("n_syrk", "<i8"), ("n_apply", "<i8"),
                   ("n_cols", "<i8"), ("n_active", "<i8"), ("sec_off", "<u8", 15), ("sec_bytes", "<u8", 15)])
SECTIONS = [("subs", SUB), ("sns", SN), ("lcp", "<i8"), ("rmap", "<i8"), ("trsm", TRSM),
            ("trsm_list", "<i4"), ("syrk", SYRK), ("syrk_list", "<i4"), ("seeds", SEED),
            ("perm", "<i4"), ("lambda", "<i4"), ("apply", APPLY), ("active", "<i4"), ("cuts", "<i4"),
            ("sblk", "<i4")]


def export_plan(plan) -> dict:
    blob = np.zeros(plan.sizes.plan_bytes, np.uint8)
    st = plan.lib.sc_export_plan(plan.h, blob.ctypes.data, blob.size)
    assert st == 0
    h = np.frombuffer(blob[:HEADER.itemsize].tobytes(), HEADER)[0]
    assert h["magic"] == 0x4C504353 and h["version"] == 1
    out = {"header": h}
    for k, (name, dt) in enumerate(SECTIONS):
        off, nb = int(h["sec_off"][k]), int(h["sec_bytes"][k])
        assert off % 256 == 0 and off + nb <= blob.size
        out[name] = np.frombuffer(blob[off:off + nb].tobytes(), dt)
    sl, il, yl = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    plan.lib.sc_workspace_layout(plan.h, ctypes.byref(sl), ctypes.byref(il), ctypes.byref(yl))
    out["ws"] = (sl.value, il.value, yl.value)
    return out


def check_bounds(T: dict, sizes, stats, tile_subs=()) -> None:
    """Every address the kernels form, against the buffer it indexes."""
    subs, sns = T["subs"], T["sns"]
    ncols = int(T["header"]["n_cols"])
    # Y offsets restart in every workspace wave: the region holds the largest wave
    ydbl = int(max([int(s["y_off"]) + int(s["ns"]) * int(s["jhi"] - s["jlo"]) for s in sns], default=0))
    assert ydbl <= int(stats.y_doubles)
    Lvals = int(sizes.L_values)
    Fd = int(sizes.F_doubles)
    assert T["ws"][2] + 8 * ydbl <= sizes.ws_bytes
    assert T["ws"][1] + 8 * ncols <= T["ws"][2]
    assert len(T["lcp"]) == ncols and (len(T["lcp"]) == 0 or (T["lcp"].min() >= 0 and T["lcp"].max() < Lvals))
    for s in sns:
        ws = s["jhi"] - s["jlo"]
        assert ws > 0 and s["ns"] > 0 and s["rs"] >= 0
        assert 0 <= s["y_off"] and s["y_off"] + s["ns"] * ws <= ydbl
        assert 0 <= s["lcp_off"] and s["lcp_off"] + s["ns"] <= ncols
        sd = subs[s["sub"]]
        assert 0 <= s["jlo"] < s["jhi"] <= sd["m"]
        assert s["c0"] + s["ns"] <= sd["n"]
        assert s["rmap_off"] + s["rs"] <= len(T["rmap"])
        nb = (s["ns"] + 31) // 32
        assert 0 <= s["cut_off"] and s["cut_off"] + nb <= len(T["cuts"])
        cuts = T["cuts"][s["cut_off"]:s["cut_off"] + nb]
        assert np.all(cuts >= s["jlo"]) and np.all(cuts <= s["jhi"]) and np.all(np.diff(cuts) >= 0)
        # every L entry the kernels read in column c0+c: rows c..ns+rs-1 of the panel
        for c in range(s["ns"]):
            g = s["lcp_off"] + c
            last = T["lcp"][g] + (s["ns"] + s["rs"] - 1 - c)
            assert last < Lvals
            if g + 1 < sd["lcp_off"] + sd["n"]:
                assert last < T["lcp"][g + 1], "panel column overruns its CSC column"
        # pruned-row targets: the source's full width must fit in the target block
        for k in range(s["rs"]):
            base = T["rmap"][s["rmap_off"] + k]
            assert 0 <= base and base + ws <= ydbl
    for e in T["seeds"]:
        assert 0 <= e["y_off"] < ydbl and np.isfinite(e["value"]) and e["value"] != 0.0
    # every (subdomain, 32-column chunk) has exactly one TRSM task, whatever the order
    chunks = sorted((int(t["sub"]), int(t["c_lo"])) for t in T["trsm"])
    assert chunks == [(i, 32 * q) for i, sd in enumerate(subs) for q in range((int(sd["m"]) + 31) // 32)]
    for t in T["trsm"]:
        sd = subs[t["sub"]]
        assert 0 < t["w"] <= 32 and t["c_lo"] + t["w"] <= sd["m"]
        assert 0 <= t["seed_lo"] <= t["seed_hi"] <= len(T["seeds"])
        lst = T["trsm_list"][t["list_off"]:t["list_off"] + t["list_len"]]
        assert len(lst) == t["list_len"] and np.all(np.diff(lst) > 0)
        for si in lst:
            s = sns[si]
            assert s["sub"] == t["sub"]
            assert max(s["jlo"], t["c_lo"]) < min(s["jhi"], t["c_lo"] + t["w"])
    for t in T["syrk"]:
        sd = subs[t["sub"]]
        if int(t["sub"]) in tile_subs:        # 128x32 tile: rows q1..q1+3 (q1 % 4 == 0), column chunk q2
            assert t["q1"] % 4 == 0 and 0 <= t["q2"] <= min(t["q1"] + 3, sd["nt"] - 1) and t["q1"] < sd["nt"]
        else:
            assert 0 <= t["q2"] <= t["q1"] < sd["nt"]
        lst = T["syrk_list"][t["list_off"]:t["list_off"] + t["list_len"]]
        assert len(lst) == t["list_len"]
    for sd in subs:
        nt = sd["nt"]
        assert sd["F_off"] + nt * (nt + 1) // 2 * 1024 <= Fd
        p = T["perm"][sd["col_off"]:sd["col_off"] + sd["m"]]
        assert np.array_equal(np.sort(p), np.arange(sd["m"]))
    assert len(T["active"]) == 0 or (T["active"].min() >= 0 and T["active"].max() < ncols)


def tc_off(r: int, k: int, R: int) -> int:
    """Byte offset of element (r, k) of an R x 32 digit block in the tcgen05
    SYRK's shared-memory layout (canonical K-major, no swizzle)."""
    return (k >> 4) * (R * 32) + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2


def check_tile_fetches(T: dict, t, yd_plane: int, S: int = 7) -> None:
    """The tcgen05 SYRK's 16-byte copies for one tile task: every source is
    inside its supernode's digit block of one plane (16-byte aligned), every
    destination inside the stage and the stage's A and B parts covered once
    (A plane by plane, B slab-major: plane d is rows 32 d .. of an S * 32-row
    operand, so that planes 0 .. S - 1 - t form the N = 32 (S - t) operand of
    A's plane t)."""
    sns = T["sns"]
    lst = T["syrk_list"][t["list_off"]:t["list_off"] + t["list_len"]]
    j1lo, j2lo = int(t["q1"]) * 32, int(t["q2"]) * 32
    j1min = max(j1lo, j2lo)
    seen_a = set(tc_off(c, 8 * kc, 128) for c in range(128) for kc in range(4))
    seen_b = set(tc_off(32 * d + c, 8 * kc, 32 * S) for d in range(S) for c in range(32) for kc in range(4))
    assert len(seen_a) == 512 and max(seen_a) + 16 <= 128 * 64 and all(o % 16 == 0 for o in seen_a)
    assert len(seen_b) == 128 * S and max(seen_b) + 16 <= S * 32 * 64 and all(o % 16 == 0 for o in seen_b)
    for ta in range(S):          # the MMA of A's plane ta reads B rows 0 .. 32 (S - ta) of each K-slab
        for ks in range(2):
            lo = ks * 32 * S * 32
            rows = [tc_off(r, 16 * ks + k, 32 * S) for r in range(32 * (S - ta)) for k in range(16)]
            assert min(rows) >= lo and max(rows) + 2 <= lo + 32 * S * 32
    for si in lst:
        s = sns[si]
        ns, ws = int(s["ns"]), int(s["jhi"] - s["jlo"])
        npad = (ns + 31) // 32 * 32
        for k0 in range(0, ns, 32):
            if j1min >= T["cuts"][s["cut_off"] + k0 // 32]:
                continue
            for base, n in ((j1lo, 128), (j2lo, 32)):
                for c in range(n):
                    j = base + c - int(s["jlo"])
                    if not (0 <= j < ws):
                        continue
                    for kc in range(4):
                        e = int(s["yd_off"]) + j * npad + k0 + 8 * kc
                        assert e % 8 == 0 and 0 <= e and e + 8 <= int(s["yd_off"]) + ws * npad <= yd_plane


def emulate_assembly(T: dict, sizes, stats, Lv: np.ndarray, tile_subs=()) -> np.ndarray:
    """Replay prep, trsm and syrk kernels in FP64; returns the F buffer.
    Subdomains in tile_subs run the 128x32 tile SYRK (tcgen05 kernel)."""
    subs, sns, lcp, rmap = T["subs"], T["sns"], T["lcp"], T["rmap"]
    invd = np.zeros(int(T["header"]["n_cols"]))
    for g in T["active"]:
        invd[g] = 1.0 / Lv[lcp[g]]
    Y = np.full(int(stats.y_doubles), np.nan)
    F = np.full(int(sizes.F_doubles), np.nan)
    # fpad
    for sd in subs:
        if sd["nt"] == 0:
            continue
        rem = sd["m"] - (sd["nt"] - 1) * 32
        if rem == 32:
            continue
        I = sd["nt"] - 1
        for J in range(I + 1):
            base = sd["F_off"] + (I * (I + 1) // 2 + J) * 1024
            for e in range(1024):
                r, c = e % 32, e // 32
                if r >= rem or (J == I and c >= rem):
                    F[base + e] = 0.0
    for t in T["trsm"]:
        lst = T["trsm_list"][t["list_off"]:t["list_off"] + t["list_len"]]
        c_hi = t["c_lo"] + t["w"]
        for si in lst:
            s = sns[si]
            a, b = max(s["jlo"], t["c_lo"]), min(s["jhi"], c_hi)
            ws = s["jhi"] - s["jlo"]
            for r in range(s["ns"]):
                o = s["y_off"] + r * ws + (a - s["jlo"])
                Y[o:o + (b - a)] = 0.0
        for e in T["seeds"][t["seed_lo"]:t["seed_hi"]]:
            Y[e["y_off"]] = e["value"]
        for si in lst:
            s = sns[si]
            a, b = max(s["jlo"], t["c_lo"]), min(s["jhi"], c_hi)
            w, ws, ns, rs = b - a, s["jhi"] - s["jlo"], s["ns"], s["rs"]
            colsh = a - s["jlo"]
            cp = lcp[s["lcp_off"]:s["lcp_off"] + ns]
            rows = lambda p: (s["y_off"] + p * ws + colsh) if p < ns else (rmap[s["rmap_off"] + p - ns] + colsh)
            for kb in range(0, ns, 32):
                kw = min(32, ns - kb)
                wk = min(b, T["cuts"][s["cut_off"] + kb // 32]) - a
                if wk <= 0:
                    continue
                for q in range(kw):      # columns past the cut must still be zero here
                    assert not np.any(Y[rows(kb + q) + wk:rows(kb + q) + w]), "nonzero past the cut"
                w_full, w = w, wk
                cps = cp[kb:kb + kw] - (kb + np.arange(kw))
                X = np.stack([Y[rows(kb + q):rows(kb + q) + w] for q in range(kw)])
                for q in range(kw):
                    X[q] = X[q] * invd[s["lcp_off"] + kb + q]
                    for r in range(q + 1, kw):
                        X[r] = X[r] - Lv[cps[q] + kb + r] * X[q]
                for q in range(kw):
                    Y[rows(kb + q):rows(kb + q) + w] = X[q]
                for p in range(kb + kw, ns + rs):
                    lrow = Lv[cps + p]
                    o = rows(p)
                    Y[o:o + w] -= lrow @ X
                w = w_full
    for t in T["syrk"]:
        sd = subs[t["sub"]]
        lst = T["syrk_list"][t["list_off"]:t["list_off"] + t["list_len"]]
        tile = int(t["sub"]) in tile_subs
        M = 128 if tile else 32
        acc = np.zeros((M, 32))
        j1lo, j2lo = t["q1"] * 32, t["q2"] * 32
        j1cut = max(j1lo, j2lo) if tile else j1lo   # the tile skips a block only if all its rows are cut
        for si in lst:
            s = sns[si]
            ws = s["jhi"] - s["jlo"]
            Ys = Y[s["y_off"]:s["y_off"] + s["ns"] * ws].reshape(s["ns"], ws).copy()
            for k0 in range(0, s["ns"], 32):          # blocks the kernel skips
                if j1cut >= T["cuts"][s["cut_off"] + k0 // 32]:
                    Ys[k0:k0 + 32] = 0.0
            A = np.zeros((s["ns"], M))
            B = np.zeros((s["ns"], 32))
            for c in range(M):
                ja = j1lo + c - s["jlo"]
                if 0 <= ja < ws:
                    A[:, c] = Ys[:, ja]
            for c in range(32):
                jb = j2lo + c - s["jlo"]
                if 0 <= jb < ws:
                    B[:, c] = Ys[:, jb]
            assert not np.isnan(A).any() and not np.isnan(B).any(), "SYRK reads unwritten Y"
            acc += A.T @ B
        perm = T["perm"][sd["col_off"]:sd["col_off"] + sd["m"]]
        for r in range(M):
            for c in range(32):
                j1, j2 = j1lo + r, j2lo + c
                if j1 < sd["m"] and j2 < sd["m"] and (j1 >= j2 if tile else (t["q1"] != t["q2"] or j1 >= j2)):
                    a, b = perm[j1], perm[j2]
                    hi, lo = max(a, b), min(a, b)
                    I, J = hi // 32, lo // 32
                    base = sd["F_off"] + (I * (I + 1) // 2 + J) * 1024
                    F[base + hi % 32 + 32 * (lo % 32)] = acc[r, c]
                    if I == J:
                        F[base + lo % 32 + 32 * (hi % 32)] = acc[r, c]
    return F


def export_dense(T: dict, F: np.ndarray, i: int) -> np.ndarray:
    sd = T["subs"][i]
    m = sd["m"]
    out = np.empty((m, m))
    for a in range(m):
        for b in range(m):
            hi, lo = max(a, b), min(a, b)
            I, J = hi // 32, lo // 32
            out[a, b] = F[sd["F_off"] + (I * (I + 1) // 2 + J) * 1024 + hi % 32 + 32 * (lo % 32)]
    return out


def check_split_layout(T: dict, sizes, stats, sub_var=None) -> dict:
    assert stats.n_waves == 1, "layout check covers single-wave plans"
    """Split-precision regions: per-supernode L digit rows (closed-form block
    bases against the prefix sums) and Y digit blocks (rows padded to 32) of
    the split subdomains are disjoint, in range and 16-byte aligned for the
    vector loads; the (supernode, block) work list is grouped by variant."""
    sns = T["sns"]
    nsub = len(T["subs"])
    sub_var = [1] * nsub if sub_var is None else list(sub_var)
    ld_end = yd_end = 0
    want = {}
    for i, s in enumerate(sns):
        v = sub_var[int(s["sub"])]
        if not v:
            continue
        ns, rs, ws = int(s["ns"]), int(s["rs"]), int(s["jhi"] - s["jlo"])
        nrow = ns + rs
        assert s["ld_off"] == ld_end, "L digit rows not contiguous"
        pre = 0
        for b, kb in enumerate(range(0, ns, 32)):
            kw = min(32, ns - kb)
            assert s["ld_off"] + b * nrow - 16 * b * (b + 1) == s["ld_off"] + pre
            pre += nrow - kb - kw
            want.setdefault(v, []).append((i, b))
        ld_end = s["ld_off"] + pre
        npad = (ns + 31) // 32 * 32
        assert s["yd_off"] == yd_end and s["yd_off"] % 32 == 0
        yd_end = s["yd_off"] + ws * npad
    assert yd_end % 32 == 0
    sb = [tuple(x) for x in T["sblk"].reshape(-1, 2).tolist()]
    assert sb == [x for v in sorted(want) for x in want[v]]
    return {"ld_rows": int(ld_end), "yd_plane": int(yd_end)}
