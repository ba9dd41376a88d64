"""GPU library vs CPU oracle: bit-exact genotypes, survivor lists, integer
statistics and the FP64 resource trajectory, on the same seeded inputs, through
the C ABI.  FP32 summaries within 1e-6 relative."""
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


def unpack(g, n_loci):
    n = g.shape[0]
    w = n_loci // 32
    words = g.reshape(n, 2, w).astype(np.uint64)
    bits = (words[..., None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return bits.reshape(n, 2, n_loci).astype(np.int64)


def run_both(w, n_gen, chunks=None):
    """Advance the oracle and the GPU population by n_gen generations (in the
    given chunks of step calls) and return both plus their stats."""
    sp = spegg()
    orc = oracle.OraclePopulation.from_workload(w)
    gpu = sp.Population.from_workload(w, stats_capacity=max(n_gen + 2, 2))
    chunks = chunks or [n_gen]
    so = [orc.step(c) for c in chunks]
    for c in chunks:
        gpu.step(c)
    so = np.concatenate(so) if so else np.zeros(0, oracle.STATS_DTYPE)
    st = gpu.state()
    sg = gpu.read_stats(1, st["gen"]) if st["gen"] else np.zeros(0, sp.STATS_DTYPE)
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


def test_single_species_workload_full_size():
    """N=10,000, L=32, 100 generations, mu=1e-4, seed 0 (graph + direct launches)."""
    w = S.single_species()
    orc, gpu, so, sg = run_both(w, 100, chunks=[1, 64, 35])
    assert len(sg) == 100
    assert_identical(orc, gpu, so, sg)


@pytest.mark.parametrize("n,n_loci,n_gen,mu,eco", [
    (3333, 64, 40, 1e-3, False),
    (20000, 128, 12, 1e-3, True),
    (5000, 256, 10, 1e-3, False),
    (4097, 256, 6, 1e-3, True),
    (6000, 32, 8, 0.05, False),    # many mutations per offspring, duplicate draws
    (3000, 128, 5, 0.02, True),
])
def test_parity_across_shapes(n, n_loci, n_gen, mu, eco):
    if eco:
        w = S.consumer_resource(n=n, n_loci=n_loci, n_gen=n_gen, mu=mu, s=1.0, K=2.0 * n, seed=5)
    else:
        w = S.single_species(n=n, n_loci=n_loci, n_gen=n_gen, mu=mu, s=2.0, seed=7, replicate=3)
    assert_identical(*run_both(w, n_gen))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2049])
@pytest.mark.parametrize("n_loci", [32, 128])
def test_tile_edges(n, n_loci):
    w = S.single_species(n=n, n_loci=n_loci, n_gen=5, mu=1e-2, s=3.0, seed=11)
    assert_identical(*run_both(w, 5))


@pytest.mark.parametrize("items", [1, 2, 4])
@pytest.mark.parametrize("n_loci", [32, 64, 128, 256])
def test_every_tiling_gives_identical_results(items, n_loci):
    sp = spegg()
    w = S.consumer_resource(n=9001, n_loci=n_loci, n_gen=6, mu=1e-3, s=1.0, K=2e5, seed=4)
    orc = oracle.OraclePopulation.from_workload(w)
    gpu = sp.Population.from_workload(w, stats_capacity=16)
    if items == 4 or (n_loci >= 128 and items == 2):
        with pytest.raises(sp.SpeggError):
            gpu.set_tiling(items)
        return
    gpu.set_tiling(items)
    assert gpu.tiling() == items
    gpu.step(3)
    gpu.set_tiling(1 if items != 1 else (2 if n_loci <= 64 else 1))
    gpu.step(3)
    assert_identical(orc, gpu, orc.step(6), gpu.read_stats(1, 6))


SHAPES = [(128, 1, 1), (128, 2, 1), (256, 1, 1), (256, 2, 1), (512, 1, 1), (512, 2, 1), (128, 1, 2), (256, 1, 2),
          (512, 1, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n_loci", [32, 64, 128, 256])
def test_every_launch_shape_gives_identical_results(shape, n_loci):
    """Threads per block, offspring per thread and lanes per offspring change
    only how the work is laid out: oracle-equal for a population whose tiles
    end mid-bucket, with a high mutation rate (the lane-pair mutation path),
    switched shape half way."""
    sp = spegg()
    block, items, lanes = shape
    w = S.consumer_resource(n=20_011, n_loci=n_loci, n_gen=6, mu=2e-3, s=1.0, K=4e5, seed=7)
    orc = oracle.OraclePopulation.from_workload(w)
    gpu = sp.Population.from_workload(w, stats_capacity=16)
    if (n_loci >= 128 and items != 1) or (n_loci <= 64 and lanes != 1):
        with pytest.raises(sp.SpeggError):
            gpu.set_launch_shape(block, items, lanes)
        return
    gpu.set_launch_shape(block, items, lanes)
    assert gpu.launch_shape() == (block, items, lanes)
    gpu.step(3)
    gpu.set_launch_shape()  # the default shape
    gpu.step(3)
    assert_identical(orc, gpu, orc.step(6), gpu.read_stats(1, 6))


@pytest.mark.parametrize("p0", [0.0, 0.3, 0.5])
def test_founders_by_philox(p0):
    w = S.single_species(n=3000, n_loci=128, n_gen=3, mu=1e-3, seed=2)
    w.p0_q32 = S.p0_threshold(p0)
    assert_identical(*run_both(w, 0))
    assert_identical(*run_both(w, 3))


def test_caller_founders():
    w = S.single_species(n=2500, n_loci=64, n_gen=4, mu=1e-3, seed=9)
    w.init_genotypes = S.genotypes_bernoulli(2500, 64, 0.2, seed=4)
    assert_identical(*run_both(w, 4))


def test_extinction():
    w = S.single_species(n=1000, n_loci=32)
    w.surv_table = S.constant_table(0)
    orc, gpu, so, sg = run_both(w, 5, chunks=[3, 2])
    assert len(sg) == 1 and sg[0]["s"] == 0 and sg[0]["status"] == 1
    assert gpu.state()["status"] == 1
    assert_identical(orc, gpu, so, sg)


def test_resource_collapse_extinction():
    w = S.consumer_resource(n=2000, n_loci=64, K=1e5, seed=3)
    w.attack = S.constant_table(2 ** 30)
    assert_identical(*run_both(w, 12))


def test_consumer_resource_full_size_first_generations():
    """N=1,000,000, L=128 with the logistic resource: two generations
    bit-exact against the oracle at full size."""
    w = S.consumer_resource()
    assert_identical(*run_both(w, 2))


def test_large_population_staged_parents():
    """N = 1,600,000, L = 128 (51 MB of parent records, above the size where a
    population stages its parents through shared memory): three generations
    bit-exact against the oracle, through a direct launch and a chunk."""
    w = S.consumer_resource(n=1_600_000)
    assert_identical(*run_both(w, 3, chunks=[1, 2]))


def test_consumer_resource_full_size_graph_path_invariants():
    """Full size through the cached-graph launches: properties that hold at
    any size, checked with numpy against the GPU's own outputs."""
    sp = spegg()
    w = S.consumer_resource()
    gpu = sp.Population.from_workload(w, stats_capacity=128)
    gpu.step(64)
    st = gpu.read_stats(1, 64)
    assert np.array_equal(st["gen"], np.arange(1, 65))
    assert np.all(st["n"] == w.n) and np.all(st["status"] == 0)
    surv = gpu.survivors()
    assert len(surv) == st[-1]["s"] == gpu.state()["S"]
    assert np.all(np.diff(surv.astype(np.int64)) > 0) and surv[-1] < w.n
    g = gpu.genotypes()
    bits = unpack(g, w.n_loci)
    raw = (bits.sum(axis=1) * w.effects.astype(np.int64)).sum(axis=1)
    last = st[-1]
    assert last["sum_raw"] == raw.sum() and last["sum_raw2"] == (raw * raw).sum()
    assert last["min_raw"] == raw.min() and last["max_raw"] == raw.max()
    assert last["sum_raw_surv"] == raw[surv].sum()
    assert last["het"] == (bits[:, 0] != bits[:, 1]).sum() and last["allele"] == bits.sum()
    v = raw + w.bias
    bins = np.where(v < 0, 0, np.minimum(v >> w.shift, 4095))
    assert last["consumption"] == w.attack[bins[surv]].astype(np.uint64).sum()


def test_two_populations_on_one_stream_are_independent():
    sp = spegg()
    w1 = S.single_species(n=4000, n_loci=64, seed=1, mu=1e-3)
    w2 = S.consumer_resource(n=3000, n_loci=128, seed=2, K=1e5, mu=1e-3)
    g1, g2 = sp.Population.from_workload(w1), sp.Population.from_workload(w2)
    o1, o2 = oracle.OraclePopulation.from_workload(w1), oracle.OraclePopulation.from_workload(w2)
    for _ in range(3):
        g1.step(5)
        g2.step(3)
    s1, s2 = o1.step(15), o2.step(9)
    assert_identical(o1, g1, s1, g1.read_stats(1, 15))
    assert_identical(o2, g2, s2, g2.read_stats(1, 9))


def test_checkpoint_resume_is_exact():
    sp = spegg()
    w = S.consumer_resource(n=5000, n_loci=128, K=1e5, mu=1e-3, seed=8)
    a = sp.Population.from_workload(w, stats_capacity=64)
    a.step(10)
    blob = a.checkpoint()
    a.step(10)
    b = sp.Population.from_workload(w, stats_capacity=64)
    b.restore(blob)
    assert b.state()["gen"] == 10
    b.step(10)
    assert np.array_equal(a.genotypes(), b.genotypes())
    assert np.array_equal(a.survivors(), b.survivors())
    assert a.read_stats(11, 10).tobytes() == b.read_stats(11, 10).tobytes()
    # rewinding the same population replays the same generations
    a.restore(blob)
    a.step(10)
    assert np.array_equal(a.genotypes(), b.genotypes())
    assert a.read_stats(11, 10).tobytes() == b.read_stats(11, 10).tobytes()


def test_stats_ring_range_and_summaries():
    sp = spegg()
    w = S.single_species(n=2000, n_loci=64, mu=1e-3)
    gpu = sp.Population.from_workload(w, stats_capacity=8)
    orc = oracle.OraclePopulation.from_workload(w)
    gpu.step(20)
    so = orc.step(20)
    with pytest.raises(sp.SpeggError) as e:
        gpu.read_stats(1, 20)
    assert e.value.code == sp.ERR_RANGE
    with pytest.raises(sp.SpeggError):
        gpu.read_stats(21, 1)
    sg = gpu.read_stats(13, 8)
    assert sg.tobytes() == so[12:].tobytes()
    one = sp.Population.from_workload(w, stats_capacity=1)
    one.step(20)
    assert one.read_stats(20, 1).tobytes() == so[19:].tobytes()
    with pytest.raises(sp.SpeggError):
        one.read_stats(19, 1)
    a = sp.summarize(sg, 64)
    b = oracle.summarize(so[12:], 64)
    assert np.allclose(a, b, rtol=1e-6, atol=0)
