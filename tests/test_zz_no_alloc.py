"""The allocation-free assembly entry point, through the C ABI.

sc_assemble_batch_static is for callers that cannot call cudaMalloc (a solver
whose memory manager already holds the free device memory, or a loop that
cannot pay cudaMalloc's device-wide synchronisation): its workspace lives in
a fixed 64 MiB array inside the library.  Its F must match the regular
sc_assemble_batch (caller workspace) within the parity tolerance, on two calls
in a row (the array keeps the first call's contents when the second starts),
and plans larger than the array must be refused before any launch.

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


@pytest.mark.parametrize("which", ["config1", "cubes"])
def test_static_matches_caller_workspace(dev, which):
    prob = synth.make_config(1) if which == "config1" else synth.cube_heat_3d(parts=2, k=6, coef_seed=3)
    fs = host.factorize_problem(prob.subdomains)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
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
