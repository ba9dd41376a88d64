"""Per-locus allele counts on the GPU (spg_set_locus_counts /
spg_read_locus_counts) against the CPU oracle: bit-exact rows for every
generation, through direct launches and cached graphs, and the rules on which
generations are kept."""
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


def sp():
    from paper_1603_09255_gb300 import spegg
    return spegg


def unpacked_counts(geno: np.ndarray, n_loci: int) -> np.ndarray:
    n = geno.shape[0]
    words = geno.reshape(n, 2, n_loci // 32).astype(np.uint64)
    bits = (words[..., None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return bits.reshape(n, 2, n_loci).sum(axis=(0, 1)).astype(np.uint32)


def oracle_rows(w, n_gen):
    orc = oracle.OraclePopulation.from_workload(w)
    rows = []
    for _ in range(n_gen):
        orc.step(1)
        rows.append(orc.locus_counts())
    return np.array(rows), orc


@pytest.mark.parametrize("n", [1, 33, 1025, 4097, 20011])
@pytest.mark.parametrize("n_loci", [32, 64, 128, 256])
def test_locus_counts_match_oracle(n, n_loci):
    """40 generations (one cached 32-generation graph and 8 direct launches),
    every row equal to the oracle's count of that generation."""
    w = S.consumer_resource(n=n, n_loci=n_loci, mu=2e-3, s=1.0, K=max(4.0 * n, 50.0), seed=31)
    gpu = sp().Population.from_workload(w, stats_capacity=64)
    gpu.set_locus_counts(True)
    gpu.step(40)
    want, orc = oracle_rows(w, 40)
    last = gpu.state()["gen"]
    assert last == orc.state()["gen"]
    got = gpu.locus_counts(1, last)
    assert np.array_equal(got, want[:last])
    gpu.close()


def test_locus_counts_one_generation_at_a_time_and_switching():
    w = S.single_species(n=3001, n_loci=128, mu=5e-3, s=1.0, seed=8)
    gpu = sp().Population.from_workload(w, stats_capacity=32)
    with pytest.raises(sp().SpeggError) as e:
        gpu.locus_counts(1, 1)
    assert e.value.code == sp().ERR_INVALID
    gpu.step(2)  # not counted
    gpu.set_locus_counts(True)
    for _ in range(3):
        gpu.step(1)
    gpu.set_locus_counts(False)
    gpu.step(2)  # not counted
    want, _ = oracle_rows(w, 7)
    assert np.array_equal(gpu.locus_counts(3, 3), want[2:5])
    for first, count in ((1, 1), (2, 2), (5, 2), (6, 1), (8, 1)):
        with pytest.raises(sp().SpeggError) as e:
            gpu.locus_counts(first, count)
        assert e.value.code == sp().ERR_RANGE
    gpu.set_locus_counts(True)  # counting again from generation 8
    gpu.step(1)
    want, _ = oracle_rows(w, 8)
    assert np.array_equal(gpu.locus_counts(8, 1), want[7:8])
    with pytest.raises(sp().SpeggError):
        gpu.locus_counts(3, 1)
    gpu.close()


def test_locus_counts_of_an_extinct_population_stay():
    w = S.single_species(n=900, n_loci=64, seed=5)
    w.surv_table = S.constant_table(0)
    gpu = sp().Population.from_workload(w, stats_capacity=16)
    gpu.set_locus_counts(True)
    gpu.step(5)  # goes extinct in its first generation; later launches change nothing
    assert gpu.state()["gen"] == 1 and gpu.state()["status"] == 1
    want, _ = oracle_rows(w, 1)
    assert np.array_equal(gpu.locus_counts(1, 1), want)
    gpu.close()


def test_locus_counts_full_size_graph_invariants():
    """N = 10^6, L = 128 through cached graphs: every row sums to the allele
    statistic of its generation and stays within 2N, and the last row is the
    count of the last generation's own records."""
    w = S.consumer_resource()
    gpu = sp().Population.from_workload(w, stats_capacity=128)
    gpu.set_locus_counts(True)
    gpu.step(64)
    rows = gpu.locus_counts(1, 64)
    st = gpu.read_stats(1, 64)
    assert np.array_equal(rows.sum(axis=1, dtype=np.uint64), st["allele"].astype(np.uint64))
    assert rows.max() <= 2 * w.n
    assert np.array_equal(rows[-1], unpacked_counts(gpu.genotypes(), w.n_loci))
    gpu.close()


def test_locus_counts_restore_and_continuous():
    w = S.single_species(n=2000, n_loci=64, mu=1e-3, seed=2)
    gpu = sp().Population.from_workload(w, stats_capacity=32)
    blob = gpu.checkpoint()
    gpu.set_locus_counts(True)
    gpu.step(4)
    gpu.restore(blob)  # back to the founders: counting restarts with generation 1
    with pytest.raises(sp().SpeggError):
        gpu.locus_counts(1, 1)
    gpu.step(3)
    want, _ = oracle_rows(w, 3)
    assert np.array_equal(gpu.locus_counts(1, 3), want)
    gpu.close()
    c = sp().Population.from_workload(S.continuous_trait(n=100, n_loci=32))
    with pytest.raises(sp().SpeggError) as e:
        c.set_locus_counts(True)
    assert e.value.code == sp().ERR_INVALID
    c.close()


def test_batch_locus_counts_match_oracle():
    """Batch members in groups of one and of two (plain, linkage map, parent
    weights, an extinct one): counts from the enabling call on, through the
    autotuner's reshaped launches and a cached graph, equal the oracle's; a
    continuous-allele member is not counted."""
    ws = [
        S.single_species(n=1000, n_loci=32, mu=2e-3, s=1.0, seed=41, replicate=0),
        S.consumer_resource(n=4097, n_loci=32, mu=2e-3, s=1.0, K=2e4, seed=41, replicate=1),
        S.single_species(n=20011, n_loci=64, mu=1e-3, s=1.0, seed=41, replicate=2),
        S.with_linkage(S.single_species(n=3000, n_loci=128, mu=1e-3, s=1.0, seed=41, replicate=3), 4, 1.0),
        S.with_linkage(S.single_species(n=33, n_loci=128, mu=1e-2, s=1.0, seed=41, replicate=4), 2, 0.5),
        S.with_weights(S.single_species(n=5000, n_loci=256, mu=1e-3, s=1.0, seed=41, replicate=5)),
        S.single_species(n=700, n_loci=64, seed=41, replicate=6),
        S.continuous_trait(n=500, n_loci=64, seed=41, replicate=7),
    ]
    ws[6].surv_table = S.constant_table(0)  # extinct in its first generation
    b = sp().Batch(ws, stats_capacity=64)
    b.set_locus_counts(True)
    ran = b.autotune(1)
    b.step(40)
    for i, w in enumerate(ws[:7]):
        gen = b.state(i)["gen"]
        want, orc = oracle_rows(w, ran + 40)
        assert gen == orc.state()["gen"], i
        assert np.array_equal(b.locus_counts(i, 1, gen), want[:gen]), i
    with pytest.raises(sp().SpeggError) as e:
        b.locus_counts(7, 1, 1)
    assert e.value.code == sp().ERR_INVALID
    b.set_locus_counts(False)
    b.step(2)
    with pytest.raises(sp().SpeggError) as e:
        b.locus_counts(0, ran + 41, 1)
    assert e.value.code == sp().ERR_RANGE
    b.close()
