"""CPU replay of the GPU implicit-apply kernel over its exported plan.

Test infrastructure for the library (not the oracle): parses the plan blob
(sci_export_plan), checks that every address the kernel forms stays inside its
buffer, and replays the kernel's FP64 arithmetic supernode block by supernode
block (the same index formulas, the same level order) with numpy, so that the
schedule and the panel addressing can be checked against the oracle without a
GPU.
"""
from __future__ import annotations

import numpy as np

HEADER = np.dtype([("magic", "<u4"), ("version", "<u4"), ("nsub", "<i4"), ("pad", "<i4"),
                   ("n_sn", "<i8"), ("n_levptr", "<i8"), ("n_rows", "<i8"), ("n_grow", "<i8"),
                   ("n_gent", "<i8"), ("n_sent", "<i8"), ("n_items", "<i8"), ("sec_off", "<u8", 8)])
SUB = np.dtype([("x_off", "<i8"), ("n", "<i4"), ("sn_lo", "<i4"), ("sn_hi", "<i4"), ("lev_lo", "<i4"),
                ("n_lev", "<i4"), ("g_lo", "<i4"), ("g_hi", "<i4"), ("s_lo", "<i4"), ("s_hi", "<i4"),
                ("n_lev_a", "<i4"), ("n_lev_b", "<i4"), ("s_mid1", "<i4"), ("s_mid2", "<i4"), ("pad", "<i4")])
SN = np.dtype([("lval", "<i8"), ("rows_off", "<i8"), ("c0", "<i4"), ("ns", "<i4"), ("rs", "<i4"),
               ("sub", "<i4")])
GROW = np.dtype([("r", "<i4"), ("e_lo", "<i4"), ("e_hi", "<i4"), ("pad", "<i4")])
GENT = np.dtype([("gj", "<i4"), ("sign", "<i4")])
SENT = np.dtype([("r", "<i4"), ("gj", "<i4"), ("sign", "<i4"), ("pad", "<i4")])
ITEM = np.dtype([("kind", "<i4"), ("n", "<i4"), ("sub", "<i4", 8)])
SECTIONS = [("subs", SUB, "nsub"), ("sns", SN, "n_sn"), ("levptr", "<i4", "n_levptr"), ("rows", "<i4", "n_rows"),
            ("grow", GROW, "n_grow"), ("gent", GENT, "n_gent"), ("sent", SENT, "n_sent"),
            ("items", ITEM, "n_items")]


def export_plan(iplan) -> dict:
    blob = iplan.export_plan()
    h = np.frombuffer(blob[:HEADER.itemsize].tobytes(), HEADER)[0]
    assert h["magic"] == 0x50494353 and h["version"] == 2
    out = {"header": h}
    for k, (name, dt, cnt) in enumerate(SECTIONS):
        off = int(h["sec_off"][k])
        n = int(h[cnt])
        nb = n * np.dtype(dt).itemsize
        assert off % 256 == 0 and off + nb <= blob.size
        out[name] = np.frombuffer(blob[off:off + nb].tobytes(), dt)
    return out


def _col_off(t: int, nr: int) -> int:
    return t * nr - t * (t - 1) // 2


def check_bounds(T: dict, sizes, L_offsets, n_dual: int) -> None:
    """Every address of the kernel against its buffer.  L_offsets: the
    concatenated-value offsets of the subdomains in input order."""
    subs, sns, lev, rows = T["subs"], T["sns"], T["levptr"], T["rows"]
    xd = (int(sizes.ws_bytes) - 256) // 8
    seen = set()
    for sd in subs:
        assert 0 <= sd["x_off"] and sd["x_off"] + sd["n"] <= xd
        assert 0 <= sd["sn_lo"] <= sd["sn_hi"] <= len(sns)
        assert 0 <= sd["lev_lo"] and sd["lev_lo"] + sd["n_lev"] < len(lev)
        assert lev[sd["lev_lo"]] == sd["sn_lo"] and lev[sd["lev_lo"] + sd["n_lev"]] == sd["sn_hi"]
        assert np.all(np.diff(lev[sd["lev_lo"]:sd["lev_lo"] + sd["n_lev"] + 1]) >= 0)
        for g in T["grow"][sd["g_lo"]:sd["g_hi"]]:
            assert 0 <= g["r"] < sd["n"] and 0 <= g["e_lo"] <= g["e_hi"] <= len(T["gent"])
        for e in T["sent"][sd["s_lo"]:sd["s_hi"]]:
            assert 0 <= e["r"] < sd["n"] and 0 <= e["gj"] < n_dual and e["sign"] in (1, -1)
        for s in range(sd["sn_lo"], sd["sn_hi"]):
            sn = sns[s]
            i = int(sn["sub"])
            seen.add(i)
            ns, rs = int(sn["ns"]), int(sn["rs"])
            nr = ns + rs
            assert ns >= 1 and rs >= 0 and 0 <= sn["c0"] and sn["c0"] + ns <= sd["n"]
            lo, hi = int(L_offsets[i]), int(L_offsets[i + 1])
            # the last entry of the last column is the highest address the kernel reads
            assert lo <= sn["lval"] and sn["lval"] + _col_off(ns - 1, nr) + (nr - (ns - 1)) <= hi
            assert 0 <= sn["rows_off"] and sn["rows_off"] + rs <= len(rows)
            R = rows[sn["rows_off"]:sn["rows_off"] + rs]
            assert np.all((R >= sn["c0"] + ns) & (R < sd["n"]))
    assert len(T["gent"]) == 0 or (T["gent"]["gj"].min() >= 0 and T["gent"]["gj"].max() < n_dual)
    assert len(seen) <= len(subs)
    # cluster items cover every subdomain exactly once
    covered = []
    for it in T["items"]:
        assert it["kind"] in (0, 1, 2) and 1 <= it["n"] <= 8
        assert it["kind"] != 0 or it["n"] == 1
        assert it["kind"] != 2 or it["n"] <= 4
        covered += [int(v) for v in it["sub"][:it["n"]]]
        if it["kind"] == 2:
            for v in it["sub"][:it["n"]]:
                check_pair_split(T, subs[int(v)])
    assert sorted(covered) == list(range(len(subs)))


def _parts(T: dict, sd) -> list:
    """Supernode index ranges of parts A, B and the top of a pair subdomain."""
    lev = T["levptr"]
    la, na, nb, n = int(sd["lev_lo"]), int(sd["n_lev_a"]), int(sd["n_lev_b"]), int(sd["n_lev"])
    return [range(lev[la], lev[la + na]), range(lev[la + na], lev[la + na + nb]),
            range(lev[la + na + nb], lev[la + n])]


def check_pair_split(T: dict, sd) -> None:
    """What the CTA pair's three barriers rely on: parts A and B are non-empty
    and touch disjoint rows of x (each part's supernodes update only their own
    part's or the top's rows; the top updates only top rows), and the scatter
    ranges [s_lo, s_mid1), [s_mid1, s_mid2), [s_mid2, s_hi) hold rows of A, B
    and the top."""
    sns, rows = T["sns"], T["rows"]
    parts = _parts(T, sd)
    assert len(parts[0]) > 0 and len(parts[1]) > 0
    owner = np.full(int(sd["n"]), -1)
    for p, rg in enumerate(parts):
        for s in rg:
            c0, ns = int(sns[s]["c0"]), int(sns[s]["ns"])
            assert np.all(owner[c0:c0 + ns] == -1)
            owner[c0:c0 + ns] = p
    for p, rg in enumerate(parts):
        for s in rg:
            sn = sns[s]
            R = rows[sn["rows_off"]:sn["rows_off"] + sn["rs"]]
            allowed = (p, 2) if p < 2 else (2,)
            assert np.all(np.isin(owner[R], allowed)), "a part updates rows of the other part"
    for p, (lo, hi) in enumerate([(sd["s_lo"], sd["s_mid1"]), (sd["s_mid1"], sd["s_mid2"]), (sd["s_mid2"], sd["s_hi"])]):
        assert sd["s_lo"] <= lo <= hi <= sd["s_hi"]
        for e in T["sent"][lo:hi]:
            assert owner[e["r"]] == p


def emulate(T: dict, sizes, Lv: np.ndarray, lam: np.ndarray, n_dual: int) -> np.ndarray:
    """The kernel's arithmetic, block by block; returns q."""
    subs, sns, lev, rows = T["subs"], T["sns"], T["levptr"], T["rows"]
    q = np.zeros(n_dual)
    for sd in subs:
        x = np.zeros(int(sd["n"]))
        for g in T["grow"][sd["g_lo"]:sd["g_hi"]]:
            ents = T["gent"][g["e_lo"]:g["e_hi"]]
            x[g["r"]] = float(np.sum(ents["sign"] * lam[ents["gj"]]))
        levels = [range(lev[sd["lev_lo"] + l], lev[sd["lev_lo"] + l + 1]) for l in range(sd["n_lev"])]
        for lv in levels:
            for s in lv:
                _forward(sns[s], Lv, rows, x)
        for lv in reversed(levels):
            for s in lv:
                _backward(sns[s], Lv, rows, x)
        for e in T["sent"][sd["s_lo"]:sd["s_hi"]]:
            q[e["gj"]] += e["sign"] * x[e["r"]]
    return q


def _panel(sn, Lv, kb, w, t_lo):
    """L(t, kb + k) for local rows t in [t_lo, nr) and k < w, read with the
    kernel's formula col_off(kb + k) + (t - kb - k)."""
    ns, rs = int(sn["ns"]), int(sn["rs"])
    nr = ns + rs
    base = int(sn["lval"])
    t = np.arange(t_lo, nr)
    P = np.empty((len(t), w))
    for k in range(w):
        P[:, k] = Lv[base + _col_off(kb + k, nr) + (t - kb - k)]
    return t, P


def _forward(sn, Lv, rows, x):
    ns, rs = int(sn["ns"]), int(sn["rs"])
    nr, c0, base = ns + rs, int(sn["c0"]), int(sn["lval"])
    R = rows[sn["rows_off"]:sn["rows_off"] + rs]
    for kb in range(0, ns, 32):
        w = min(32, ns - kb)
        xi = x[c0 + kb:c0 + kb + w].copy()
        for k in range(w):
            d = Lv[base + _col_off(kb + k, nr)]
            assert d > 0
            xi[k] = xi[k] * (1.0 / d)
            for i in range(k + 1, w):
                xi[i] -= Lv[base + _col_off(kb + k, nr) + (i - k)] * xi[k]
        x[c0 + kb:c0 + kb + w] = xi
        t, P = _panel(sn, Lv, kb, w, kb + w)
        acc = P @ xi
        own = t < ns
        x[c0 + t[own]] -= acc[own]
        np.subtract.at(x, R[t[~own] - ns], acc[~own])


def _backward(sn, Lv, rows, x):
    ns, rs = int(sn["ns"]), int(sn["rs"])
    nr, c0, base = ns + rs, int(sn["c0"]), int(sn["lval"])
    R = rows[sn["rows_off"]:sn["rows_off"] + rs]
    for kb in range(((ns - 1) // 32) * 32, -1, -32):
        w = min(32, ns - kb)
        t, P = _panel(sn, Lv, kb, w, kb + w)
        z = np.where(t < ns, x[np.minimum(c0 + t, len(x) - 1)], 0.0)
        z[t >= ns] = x[R[t[t >= ns] - ns]]
        rhs = x[c0 + kb:c0 + kb + w] - P.T @ z
        for i in range(w - 1, -1, -1):
            rhs[i] *= 1.0 / Lv[base + _col_off(kb + i, nr)]
            for k in range(i):
                rhs[k] -= Lv[base + _col_off(kb + k, nr) + (i - k)] * rhs[i]
        x[c0 + kb:c0 + kb + w] = rhs
