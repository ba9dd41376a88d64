"""Linkage maps on the GPU (the gamete masks of spg_pop_desc.map_morgans)
against the CPU oracle: bit-exact statistics, genotypes, survivor lists and
state, through the C ABI, for several map shapes and locus counts."""
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


def random_map(L, chromosomes, total, seed):
    """Chromosome starts at random loci, random interval lengths summing to
    `total` Morgans."""
    rng = np.random.default_rng(seed)
    m = rng.random(L)
    starts = np.sort(rng.choice(np.arange(1, L), chromosomes - 1, replace=False))
    m[0] = 0.0
    m[starts] = 0.0
    m *= total / m.sum()
    m[0] = -1.0
    m[starts] = -1.0
    return m


def maps(L):
    zero = np.zeros(L)
    zero[0] = -1.0
    return {
        "one chromosome 1 M": S.linkage_map(L, 1, 1.0),
        "4 chromosomes 2 M": S.linkage_map(L, 4, 2.0) if L >= 4 else S.linkage_map(L, 1, 2.0),
        "every locus a chromosome": np.full(L, -1.0) if L <= 96 else random_map(L, 96, 3.0, 1),
        "zero length": zero,
        "random 15.9 M": random_map(L, min(12, L // 4), 15.9, L),
    }


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
@pytest.mark.parametrize("kind", ["one chromosome 1 M", "4 chromosomes 2 M", "every locus a chromosome",
                                  "zero length", "random 15.9 M"])
def test_linked_population_matches_oracle(n_loci, kind):
    w = S.single_species(n=2500, n_loci=n_loci, mu=1e-3, seed=n_loci)
    w = dataclasses.replace(w, map_morgans=maps(n_loci)[kind])
    orc, gpu, so, sg = run_both(w, 12)
    assert_identical(orc, gpu, so, sg)


@pytest.mark.parametrize("n", [1, 33, 257, 40001])
def test_linked_edges_and_ecology(n):
    w = S.with_linkage(S.consumer_resource(n=n, n_loci=128, K=1e5, mu=1e-3), 4, 1.5)
    orc, gpu, so, sg = run_both(w, 8)
    assert_identical(orc, gpu, so, sg)


def test_linked_full_size_two_generations():
    """The measured configuration (10^6 offspring, L = 128, 4 chromosomes of
    1 Morgan) bit-exact for two generations."""
    w = S.with_linkage(S.consumer_resource(), 4, 1.0)
    orc, gpu, so, sg = run_both(w, 2)
    assert_identical(orc, gpu, so, sg)


def test_linkage_map_validation_through_the_abi():
    sp = spegg()
    w = S.single_species(n=100, n_loci=64)
    for bad in (np.full(64, 1.0), np.full(64, np.nan)):
        with pytest.raises(sp.SpeggError):
            sp.Population.from_workload(dataclasses.replace(w, map_morgans=bad))
    p = sp.Population.from_workload(dataclasses.replace(w, map_morgans=S.linkage_map(64, 2, 1.0)))
    with pytest.raises(sp.SpeggError):
        p.set_tiling(2)
    # batches and served jobs take a map and check it like a population
    with pytest.raises(sp.SpeggError):
        sp.Batch([w, dataclasses.replace(w, map_morgans=np.full(64, np.nan))])
    srv = sp.Server()
    with pytest.raises(sp.SpeggError):
        srv.submit(dataclasses.replace(w, map_morgans=np.full(64, 1.0)), 4)
    srv.close()
    sp.Batch([dataclasses.replace(w, map_morgans=S.linkage_map(64, 2, 1.0))]).close()
