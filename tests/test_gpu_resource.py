"""Beverton-Holt resource with a growth rate drawn each generation on the
GPU against the CPU oracle: bit-exact resource trajectory (FP64), statistics,
genotypes and state through the C ABI, alone, as a batch member and as a
served job."""
import dataclasses

import numpy as np
import pytest

import oracle
import spegg_synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09255_gb300 import build
    build.build()


def spegg():
    from paper_1603_09255_gb300 import spegg as m
    return m


@pytest.mark.parametrize("r,r_sd,n_loci", [(2.0, 0.0, 64), (2.0, 0.3, 128), (1.6, 0.5, 32), (3.0, 0.1, 256)])
def test_beverton_holt_matches_oracle(r, r_sd, n_loci):
    sp = spegg()
    w = S.with_beverton_holt(S.consumer_resource(n=20000, n_loci=n_loci, K=2e5, mu=1e-3, seed=n_loci), r, r_sd)
    orc = oracle.OraclePopulation.from_workload(w)
    gpu = sp.Population.from_workload(w, stats_capacity=64)
    so = orc.step(40)
    gpu.step(40)
    sg = gpu.read_stats(1, 40)
    for name in so.dtype.names:
        assert np.array_equal(so[name], sg[name]), name
    assert np.array_equal(orc.genotypes(), gpu.genotypes())
    a, b = orc.state(), gpu.state()
    for k in ("gen", "S", "status", "f", "R"):
        assert a[k] == b[k], (k, a[k], b[k])


def test_beverton_holt_batch_member_and_served_job():
    sp = spegg()
    ws = [S.with_beverton_holt(S.consumer_resource(n=3000 + 1000 * i, n_loci=64, K=1e5, mu=1e-3, seed=i,
                                                   replicate=i), 2.0, 0.25) for i in range(3)]
    batch = sp.Batch(ws, stats_capacity=32)
    batch.step(20)
    for i, w in enumerate(ws):
        so = oracle.OraclePopulation.from_workload(w).step(20)
        sg = batch.read_stats(i, 1, 20)
        for name in so.dtype.names:
            assert np.array_equal(so[name], sg[name]), (i, name)
    srv = sp.Server(memory_budget=1 << 30, max_resident=4, gens_per_tick=8)
    job = srv.submit(ws[1], 20, 0.0)
    srv.drain()
    so = oracle.OraclePopulation.from_workload(ws[1]).step(20)
    sg = srv.job_stats(job, 1, 20)
    for name in so.dtype.names:
        assert np.array_equal(so[name], sg[name]), name


def test_resource_model_validation():
    sp = spegg()
    w = S.consumer_resource(n=100, n_loci=32, K=1e5)
    p = sp.Population.from_workload(dataclasses.replace(w, eco_model=0, eco_r_sd=0.0))
    with pytest.raises(sp.SpeggError):
        p.set_ecology(w.eco_r, w.eco_K, w.eco_R0, w.eco_R_half, w.attack, model=2)
    with pytest.raises(sp.SpeggError):
        p.set_ecology(w.eco_r, w.eco_K, w.eco_R0, w.eco_R_half, w.attack, model=0, r_sd=0.1)
    with pytest.raises(sp.SpeggError):
        p.set_ecology(w.eco_r, w.eco_K, w.eco_R0, w.eco_R_half, w.attack, model=1, r_sd=-1.0)
