"""The allocation-free assembly entry point, through the C ABI.

sc_assemble_batch_static is for callers that cannot call cudaMalloc (a solver
whose memory manager already holds the free device memory, or a loop that
cannot pay cudaMalloc's device-wide synchronisation): its workspace lives in
a fixed 64 MiB array inside the library.  Its F must match the regular
sc_assemble_batch (caller workspace) within the parity tolerance and bit for
bit (the same kernels run on the same inputs), on two calls in a row (the
array keeps the first call's contents when the second starts), for FP64,
split-precision, persistent-queue and multi-wave plans; a non-positive pivot
must come back as SC_ERR_NOT_SPD from the call itself, and plans larger than
the array or a misaligned F must be refused before any launch.

This file is named so that pytest collects it last; it builds everything it
needs itself, so it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_2509_21037_gb300 import abi, host, sc

pytestmark = pytest.mark.gpu
TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _static_call(plan, Lv, F, stream=None):
    s = None if stream is None else stream.cuda_stream
    return plan.lib.sc_assemble_batch_static(plan.h, Lv.data_ptr(), F.data_ptr(), s)


def _plan(fs, n_dual, dev, variant):
    """The plan forms the static entry point must cover: default FP64, a
    split-precision variant (its digit-plane workspace regions), the
    persistent work queue (its counters in the status area) and a workspace
    bound that forces several waves."""
    nsub = len(fs)
    if variant == "fp64":
        return sc.Plan(fs, n_dual).upload(dev)
    if variant == "split5":
        return sc.Plan(fs, n_dual, sub_slices=[5] * nsub).upload(dev)
    if variant == "persistent":
        return sc.Plan(fs, n_dual, persistent=True).upload(dev)
    one = sc.Plan(fs, n_dual)
    plan = sc.Plan(fs, n_dual, ws_limit=one.sizes.ws_bytes // 3).upload(dev)
    assert plan.stats.n_waves >= 3
    return plan


@pytest.mark.parametrize("which,variant", [("config1", "fp64"), ("cubes", "fp64"), ("cubes", "split5"),
                                           ("cubes", "persistent"), ("cubes", "waves")])
def test_static_matches_caller_workspace(dev, which, variant):
    prob = synth.make_config(1) if which == "config1" else synth.cube_heat_3d(parts=2, k=6, coef_seed=3)
    fs = host.factorize_problem(prob.subdomains)
    plan = _plan(fs, prob.n_dual, dev, variant)
    assert plan.sizes.ws_bytes <= abi_static_bytes()
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F_ref = plan.new_F(dev)
    plan.assemble(Lv, F_ref)
    assert plan.device_status() == abi.SC_OK
    ref = [plan.export(F_ref, i).cpu().numpy() for i in range(plan.nsub)]
    for call in range(2):                      # two calls in a row share the array
        F = plan.new_F(dev)
        F.fill_(float("nan"))
        st = _static_call(plan, Lv, F)
        assert st == abi.SC_OK, plan.lib.sc_last_error(plan.h).decode()
        for i in range(plan.nsub):
            got = plan.export(F, i).cpu().numpy()
            assert np.isfinite(got).all()
            assert oracle.relative_frobenius(got, ref[i]) <= TOL, f"call {call}, subdomain {i}"
        # the same kernels on the same inputs: the whole F buffer is bit-identical
        assert torch.equal(F, F_ref), f"call {call}: static F differs from the caller-workspace F"


def test_static_reports_not_spd_then_recovers(dev):
    """The status word is read back by the static call itself: a negated
    diagonal entry of L gives SC_ERR_NOT_SPD, and the next call with the
    original values (same shared array) gives SC_OK and the right F."""
    prob = synth.cube_heat_3d(parts=2, k=4)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    good = sc.concat_L_values(fs)
    bad = good.copy()
    c = fs[3].n - 1                             # the root column of subdomain 3: always active
    bad[plan.L_offsets[3] + fs[3].L.colptr[c]] *= -1.0
    F = plan.new_F(dev)
    st = _static_call(plan, torch.from_numpy(bad).to(dev), F)
    assert st == abi.SC_ERR_NOT_SPD
    Lv = torch.from_numpy(good).to(dev)
    st = _static_call(plan, Lv, F)
    assert st == abi.SC_OK, plan.lib.sc_last_error(plan.h).decode()
    F_ref = plan.new_F(dev)
    plan.assemble(Lv, F_ref)
    assert plan.device_status() == abi.SC_OK
    assert torch.equal(F, F_ref)


def test_static_rejects_misaligned_F(dev):
    prob = synth.make_config(1)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    raw = torch.empty(plan.sizes.F_doubles * 8 + 16, dtype=torch.uint8, device=dev)
    st = plan.lib.sc_assemble_batch_static(plan.h, Lv.data_ptr(), raw.data_ptr() + 4, None)
    assert st == abi.SC_ERR_INVALID_ARG
    assert "misaligned" in plan.lib.sc_last_error(plan.h).decode()


def test_static_rejects_plan_beyond_scratch(dev):
    prob = synth.make_config(2)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    assert plan.sizes.ws_bytes > abi_static_bytes()
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    F = plan.new_F(dev)
    st = _static_call(plan, Lv, F)
    assert st == abi.SC_ERR_OOM
    assert "static scratch" in plan.lib.sc_last_error(plan.h).decode()


def abi_static_bytes():
    return 64 << 20
