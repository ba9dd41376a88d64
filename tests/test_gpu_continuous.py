"""Continuous allelic values on the GPU (spg_pop_desc.allele_model = 1)
against the CPU oracle: bit-exact int16 values, statistics, survivor lists
and state through the C ABI."""
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
    assert np.array_equal(orc.values(), gpu.values())
    assert np.array_equal(orc.survivors(), gpu.survivors())
    a, b = orc.state(), gpu.state()
    for k in ("gen", "S", "status", "f", "R"):
        assert a[k] == b[k], (k, a[k], b[k])


def with_ecology(w, K=1e6):
    return dataclasses.replace(w, eco_r=0.5, eco_K=K, eco_R0=K / 2, eco_R_half=K / 10,
                               attack=S.attack_table(w.bias, w.shift))


@pytest.mark.parametrize("n_loci", [32, 64, 128, 256])
@pytest.mark.parametrize("mu,mut_sd,env_sd", [(1e-2, 0.1, 0.2), (0.1, 0.5, 0.0), (1e-3, 0.0, 0.3)])
def test_continuous_matches_oracle(n_loci, mu, mut_sd, env_sd):
    w = S.continuous_trait(n=2500, n_loci=n_loci, mu=mu, mut_sd=mut_sd, env_sd=env_sd, seed=n_loci)
    orc, gpu, so, sg = run_both(w, 12)
    assert_identical(orc, gpu, so, sg)


def test_continuous_from_caller_values():
    n, L = 3000, 64
    rng = np.random.default_rng(3)
    v = rng.integers(-300, 300, size=(n, 2, L)).astype(np.int16)
    w = dataclasses.replace(S.continuous_trait(n=n, n_loci=L, mu=0.02, seed=2), init_values=v)
    orc, gpu, so, sg = run_both(w, 10)
    assert_identical(orc, gpu, so, sg)


@pytest.mark.parametrize("n", [1, 33, 257, 20001])
def test_continuous_edges_with_ecology(n):
    w = with_ecology(S.continuous_trait(n=n, n_loci=128, mu=5e-3, seed=7), K=max(n, 10) * 30.0)
    orc, gpu, so, sg = run_both(w, 8)
    assert_identical(orc, gpu, so, sg)


def test_continuous_checkpoint_resume():
    sp = spegg()
    w = S.continuous_trait(n=4000, n_loci=128, mu=1e-2, seed=9)
    a = sp.Population.from_workload(w, stats_capacity=64)
    a.step(6)
    blob = a.checkpoint()
    a.step(5)
    b = sp.Population.from_workload(w, stats_capacity=64)
    b.restore(blob)
    b.step(5)
    assert np.array_equal(a.values(), b.values())
    sa, sb = a.read_stats(7, 5), b.read_stats(7, 5)
    for name in sa.dtype.names:
        assert np.array_equal(sa[name], sb[name]), name


def test_continuous_validation_through_the_abi():
    sp = spegg()
    w = S.continuous_trait(n=100, n_loci=64)
    with pytest.raises(sp.SpeggError):
        sp.Population.from_workload(dataclasses.replace(w, allele_model=2))
    with pytest.raises(sp.SpeggError):
        sp.Population.from_workload(dataclasses.replace(w, map_morgans=S.linkage_map(64, 2, 1.0)))
    with pytest.raises(sp.SpeggError):
        sp.Population.from_workload(dataclasses.replace(w, mut_sd=100.0))
    # batch members and served jobs are checked alike
    with pytest.raises(sp.SpeggError):
        sp.Batch([w, dataclasses.replace(w, mut_sd=100.0)])
    srv = sp.Server()
    with pytest.raises(sp.SpeggError):
        srv.submit(dataclasses.replace(w, map_morgans=S.linkage_map(64, 2, 1.0)), 4)
    srv.close()
    sp.Batch([w]).close()


def test_continuous_full_size_two_generations():
    """The measured continuous-allele configuration (N = 10^6, L = 128,
    mu 1e-3, mutation sd 0.05, environmental sd 0.2) for two generations."""
    w = S.continuous_trait(n=1_000_000, n_loci=128, mu=1e-3, mut_sd=0.05, env_sd=0.2)
    orc, gpu, so, sg = run_both(w, 2)
    assert_identical(orc, gpu, so, sg)
