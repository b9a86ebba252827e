"""GPU checks of the CPU/GPU pipeline of the numeric stage
(include/sc_pipeline.h): host factorisation of chunk c+1 overlapped with the
copy and assembly of chunk c gives the same F as the direct path, bit for
bit, and the oracle's F within 1e-12."""
import numpy as np
import pytest

import oracle
import synth
from paper_2509_21037_gb300 import abi, host, pipeline, sc

pytestmark = pytest.mark.gpu
TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("nchunks", [1, 3, 5])
def test_pipeline_matches_direct_and_oracle(nchunks, dev):
    prob = synth.cube_heat_3d(2, 6, coef_seed=7)           # every subdomain its own K
    fs = host.factorize_problem(prob.subdomains)
    pipe = pipeline.Pipeline(prob.subdomains, fs, prob.n_dual, nchunks=nchunks, device=dev, nthreads=3)
    t = pipe.run()
    assert t["wall_ms"] > 0 and t["h2d_bytes"] == 8 * sum(f.L.values.size for f in fs)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    F = plan.new_F(dev)
    plan.assemble(torch.from_numpy(sc.concat_L_values(fs)).to(dev), F)
    assert plan.device_status() == abi.SC_OK
    Fo = oracle.dual_operators(prob.subdomains)
    for i in range(len(fs)):
        Fp = pipe.export(i).cpu().numpy()
        assert np.array_equal(Fp, plan.export(F, i).cpu().numpy()), f"subdomain {i} differs from the direct path"
        assert oracle.relative_frobenius(Fp, Fo[i]) <= TOL


def test_pipeline_new_values_same_patterns(dev):
    """The numeric stage reruns with new K values (same patterns): K -> 4 K
    gives F -> F / 4 on every subdomain."""
    prob = synth.cube_heat_3d(2, 5, coef_seed=2)
    fs = host.factorize_problem(prob.subdomains)
    pipe = pipeline.Pipeline(prob.subdomains, fs, prob.n_dual, nchunks=2, device=dev, nthreads=2)
    pipe.run()
    F1 = [pipe.export(i).cpu().numpy() for i in range(len(fs))]
    scaled = [synth.Subdomain(K=sd.K * 4.0, fixed=sd.fixed, Bt=sd.Bt, lambda_map=sd.lambda_map, grid=sd.grid,
                              ndpn=sd.ndpn, key=None) for sd in prob.subdomains]
    pipe2 = pipeline.Pipeline(scaled, fs, prob.n_dual, nchunks=2, device=dev, nthreads=2)
    pipe2.run()
    for i in range(len(fs)):
        sd = prob.subdomains[i]
        F4 = pipe2.export(i).cpu().numpy()
        # fixed dofs keep a unit diagonal, so compare on the columns of free dofs only
        Bt = sd.Bt.tocsc()
        cols = [j for j in range(Bt.shape[1]) if not np.isin(Bt.indices[Bt.indptr[j]:Bt.indptr[j + 1]], sd.fixed).any()]
        assert np.allclose(F4[np.ix_(cols, cols)] * 4.0, F1[i][np.ix_(cols, cols)], rtol=1e-13, atol=1e-15)


def test_pipeline_reports_not_spd(dev):
    prob = synth.cube_heat_3d(2, 4)
    fs = host.factorize_problem(prob.subdomains)
    bad = list(prob.subdomains)
    sd = bad[3]
    bad[3] = synth.Subdomain(K=-sd.K, fixed=sd.fixed, Bt=sd.Bt, lambda_map=sd.lambda_map, grid=sd.grid,
                             ndpn=sd.ndpn, key=None)
    pipe = pipeline.Pipeline(bad, fs, prob.n_dual, nchunks=2, device=dev, nthreads=2)
    with pytest.raises(sc.SCError, match="SC_ERR_NOT_SPD"):
        pipe.run()
