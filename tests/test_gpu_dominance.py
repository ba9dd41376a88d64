"""Dominance deviations on the GPU (spg_pop_desc.dominance) against the CPU
oracle: bit-exact statistics, genotypes, survivor lists and state through the
C ABI, for single populations, weighted parents and batch members."""
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
def test_dominance_matches_oracle(n_loci):
    w = S.with_dominance(S.single_species(n=2500, n_loci=n_loci, mu=1e-3, seed=n_loci), sd=0.2)
    orc, gpu, so, sg = run_both(w, 12)
    assert_identical(orc, gpu, so, sg)


def test_constant_dominance_deviation():
    """Every locus the same deviation: no planes, only the d_min term."""
    w = S.single_species(n=3000, n_loci=64, mu=1e-3, seed=3)
    w = dataclasses.replace(w, dominance=np.full(64, 7, np.int16), bias=w.bias, shift=w.shift + 1)
    w.surv_table = S.stabilizing_table(w.bias, w.shift, 0.5)
    orc, gpu, so, sg = run_both(w, 8)
    assert_identical(orc, gpu, so, sg)


def test_dominance_with_ecology_and_weighted_parents():
    w = S.with_weights(S.with_dominance(S.consumer_resource(n=20000, n_loci=128, K=1e6, mu=1e-3)))
    orc, gpu, so, sg = run_both(w, 8)
    assert_identical(orc, gpu, so, sg)


def test_zero_dominance_equals_additive_on_the_gpu():
    sp = spegg()
    w = S.single_species(n=5000, n_loci=128, mu=1e-3, seed=6)
    a = sp.Population.from_workload(w, stats_capacity=16)
    b = sp.Population.from_workload(dataclasses.replace(w, dominance=np.zeros(128, np.int16)), stats_capacity=16)
    a.step(10)
    b.step(10)
    assert np.array_equal(a.genotypes(), b.genotypes())
    sa, sb = a.read_stats(1, 10), b.read_stats(1, 10)
    for name in sa.dtype.names:
        assert np.array_equal(sa[name], sb[name]), name


def test_dominance_in_a_batch():
    sp = spegg()
    ws = [S.with_dominance(S.single_species(n=1500 + 700 * i, n_loci=L, mu=1e-3, seed=i, replicate=i), sd=0.15)
          for i, L in enumerate((32, 64, 128, 64))]
    batch = sp.Batch(ws, stats_capacity=16)
    batch.step(9)
    for i, w in enumerate(ws):
        orc = oracle.OraclePopulation.from_workload(w)
        so = orc.step(9)
        sg = batch.read_stats(i, 1, 9)
        for name in so.dtype.names:
            assert np.array_equal(so[name], sg[name]), (i, name)
        assert np.array_equal(orc.genotypes(), batch.genotypes(i))


def test_dominance_full_size_two_generations():
    """The measured dominance configuration (consumer-resource population,
    N = 10^6, L = 128, deviations Q8(N(0, 0.1))) for two generations."""
    w = S.with_dominance(S.consumer_resource())
    orc, gpu, so, sg = run_both(w, 2)
    assert_identical(orc, gpu, so, sg)
