"""Weighted parents on the GPU (spg_pop_desc.mother_weights/father_weights)
against the CPU oracle: bit-exact statistics, genotypes, survivor lists and
state through the C ABI, including the 64-proposal fallback, linkage maps,
ecology and checkpoint/resume."""
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


def run_both(w, n_gen):
    sp = spegg()
    orc = oracle.OraclePopulation.from_workload(w)
    gpu = sp.Population.from_workload(w, stats_capacity=n_gen + 2)
    so = orc.step(n_gen)
    gpu.step(n_gen)
    sg = gpu.read_stats(1, gpu.state()["gen"])
    return orc, gpu, so, sg


def assert_identical(orc, gpu, so, sg):
    assert len(so) == len(sg)
    for name in so.dtype.names:
        assert np.array_equal(so[name], sg[name]), name
    assert np.array_equal(orc.genotypes(), gpu.genotypes())
    assert np.array_equal(orc.survivors(), gpu.survivors())
    a, b = orc.state(), gpu.state()
    for k in ("gen", "S", "status", "f", "R"):
        assert a[k] == b[k], (k, a[k], b[k])


@pytest.mark.parametrize("n_loci", [32, 64, 128, 256])
def test_weighted_population_matches_oracle(n_loci):
    w = S.with_weights(S.single_species(n=2500, n_loci=n_loci, mu=1e-3, seed=n_loci), slope=1.5)
    orc, gpu, so, sg = run_both(w, 12)
    assert_identical(orc, gpu, so, sg)


@pytest.mark.parametrize("n_loci", [64, 256])
def test_weighted_and_linked(n_loci):
    w = S.with_linkage(S.with_weights(S.single_species(n=3000, n_loci=n_loci, mu=1e-3, seed=5)), 4, 2.0)
    orc, gpu, so, sg = run_both(w, 10)
    assert_identical(orc, gpu, so, sg)


def test_rare_acceptance_exercises_the_proposal_bound():
    """Only the top bins carry weight: most proposals are rejected and many
    parents come from the last of the 64 proposals."""
    w = S.single_species(n=4000, n_loci=64, mu=1e-3, seed=2)
    mw = np.zeros(4096, np.uint32)
    mw[w.bias >> w.shift:] = 1  # bins above the zero-trait bin
    mw[-600:] = 1000
    fw = np.ones(4096, np.uint32)
    fw[:10] = 5
    w = dataclasses.replace(w, mother_weights=mw, father_weights=fw)
    orc, gpu, so, sg = run_both(w, 8)
    assert_identical(orc, gpu, so, sg)


@pytest.mark.parametrize("n", [1, 33, 257])
def test_weighted_edges_with_ecology(n):
    w = S.with_weights(S.consumer_resource(n=n, n_loci=128, K=1e5, mu=1e-3))
    orc, gpu, so, sg = run_both(w, 8)
    assert_identical(orc, gpu, so, sg)


def test_weighted_checkpoint_resume_is_exact():
    sp = spegg()
    w = S.with_weights(S.single_species(n=3000, n_loci=128, mu=1e-3, seed=8))
    a = sp.Population.from_workload(w, stats_capacity=64)
    a.step(5)
    blob = a.checkpoint()
    a.step(7)
    b = sp.Population.from_workload(w, stats_capacity=64)
    b.restore(blob)
    b.step(7)
    assert np.array_equal(a.genotypes(), b.genotypes())
    assert np.array_equal(a.survivors(), b.survivors())
    sa, sb = a.read_stats(6, 7), b.read_stats(6, 7)
    for name in sa.dtype.names:
        assert np.array_equal(sa[name], sb[name]), name


def test_weighted_full_size_two_generations():
    w = S.with_weights(S.consumer_resource())
    orc, gpu, so, sg = run_both(w, 2)
    assert_identical(orc, gpu, so, sg)


def test_weight_validation_through_the_abi():
    sp = spegg()
    w = S.single_species(n=100, n_loci=64)
    with pytest.raises(sp.SpeggError):
        sp.Population.from_workload(dataclasses.replace(w, mother_weights=np.zeros(4096, np.uint32)))
    ok = S.with_weights(w)
    p = sp.Population.from_workload(ok)
    with pytest.raises(sp.SpeggError):
        p.set_tiling(4)
    zero = dataclasses.replace(w, mother_weights=np.zeros(4096, np.uint32))
    with pytest.raises(sp.SpeggError):
        sp.Batch([ok, zero])
    srv = sp.Server()
    with pytest.raises(sp.SpeggError):
        srv.submit(zero, 4)
    srv.close()
    sp.Batch([ok]).close()
