"""Seeded random corruptions of valid inputs through every host-side entry
point that checks them: sc_plan and sci_plan (one subdomain descriptor), and
both host implicit applies (L and B^T patterns, multiplier map).  Each call
must return a status -- the two planners the same one, the two host applies
the same verdict -- and never crash or read out of bounds."""
import ctypes

import numpy as np
import pytest

import synth
from paper_2509_21037_gb300 import _native, abi, host

import test_abi as ta

N_CASES = 60
_SPECIALS = [-1, 0, 1, 2, 2**31 - 1, -2**31]


@pytest.fixture(scope="module")
def batch():
    prob = synth.cube_heat_3d(2, 3)
    return prob, host.factorize_problem(prob.subdomains)


def _corrupt(rng, a):
    a = a.copy()
    for _ in range(int(rng.integers(1, 4))):
        i = int(rng.integers(0, len(a)))
        if a.dtype == np.int8:
            a[i] = int(rng.choice([-128, -1, 0, 1, 2]))
        else:
            info = np.iinfo(a.dtype)
            v = int(rng.choice(_SPECIALS + [len(a), int(a[i]) + 1, int(a[i]) - 1]))
            a[i] = min(max(v, info.min), info.max)
    return a


def test_planners_reject_or_accept_consistently(batch):
    prob, fs = batch
    rng = np.random.default_rng(2024)
    lib = _native.sc_lib()
    seen = set()
    for _ in range(N_CASES):
        f = fs[int(rng.integers(0, len(fs)))]
        field = ["colptr", "rowind", "btc", "btr", "sign", "lam", "n", "m"][int(rng.integers(0, 8))]
        src = {"colptr": f.L.colptr, "rowind": f.L.rowind, "btc": f.bt_colptr, "btr": f.bt_rowind,
               "sign": f.bt_sign, "lam": f.lambda_map}
        if field in src:
            over = {field: _corrupt(rng, src[field])}
        elif field == "n":
            over = {"n": int(rng.choice([0, 1, f.n - 1, f.n + 1, -1]))}
        else:
            over = {"m": int(rng.choice([0, 1, f.m - 1, f.m + 1, -1]))}
        keep = []
        d = ta._desc_from(f, keep, **over)
        st, msg = ta._plan_raw([d], prob.n_dual)
        h = ctypes.c_void_p()
        st2 = lib.sci_plan(ctypes.byref(h), 1, (abi.SubdomainDesc * 1)(d), prob.n_dual, None)
        lib.sci_destroy(h)
        assert st in (abi.SC_OK, abi.SC_ERR_INVALID_ARG) and st == st2, (field, st, st2, msg)
        seen.add(st)
    assert seen == {abi.SC_OK, abi.SC_ERR_INVALID_ARG}


def test_host_implicit_applies_agree_on_corrupted_inputs(batch):
    prob, fs = batch
    rng = np.random.default_rng(77)
    verdicts = set()
    for _ in range(N_CASES):
        i = int(rng.integers(0, len(fs)))
        f = fs[i]
        arrs = {"colptr": f.L.colptr, "rowind": f.L.rowind, "btc": f.bt_colptr, "btr": f.bt_rowind,
                "lam": f.lambda_map}
        field = list(arrs)[int(rng.integers(0, len(arrs)))]
        arrs = dict(arrs, **{field: _corrupt(rng, arrs[field])})
        L = host.HostFactor(f.L.n, arrs["colptr"], arrs["rowind"], f.L.values, f.L.perm)
        bad = host.FactoredSubdomain(L=L, bt_colptr=arrs["btc"], bt_rowind=arrs["btr"], bt_sign=f.bt_sign,
                                     lambda_map=arrs["lam"])
        subs = fs[:i] + [bad] + fs[i + 1:]
        out = []
        for planned in (False, True):
            try:
                q = host.ImplicitApply(subs, prob.n_dual, planned=planned)(np.ones(prob.n_dual), threads=2)
                out.append(q)
            except RuntimeError:
                out.append(None)
        assert (out[0] is None) == (out[1] is None), field
        if out[0] is not None:
            assert np.allclose(out[0], out[1], rtol=1e-12, atol=1e-12 * np.abs(out[0]).max())
        verdicts.add(out[0] is None)
    assert verdicts == {True, False}
