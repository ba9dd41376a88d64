"""Spatial community on the GPU (spg_space_*) against the CPU oracle: every
deme's records and ages, and every statistics record, bit for bit."""
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


def assert_same(gpu, orc, steps):
    so = orc.step(steps)
    t = gpu.state()["t"]
    sg = gpu.read_stats(t - steps + 1, steps)
    for name in so.dtype.names:
        assert np.array_equal(so[name], sg[name]), name
    assert np.array_equal(gpu.sizes(), orc.sizes())
    for s in range(gpu.ns):
        for p in range(gpu.c.patches):
            rg, ag = gpu.deme(s, p)
            ro, ao = orc.deme(s, p)
            assert np.array_equal(ag, ao), (s, p)
            assert np.array_equal(rg, ro), (s, p)


@pytest.mark.parametrize("X,Y,n0,L,steps,disp", [
    (4, 4, 120, 64, 8, 0.05),
    (3, 5, 60, 256, 6, 0.3),
    (1, 1, 500, 32, 10, 0.5),
    (2, 1, 80, 128, 8, 0.9),     # neighbours coincide on a 2 x 1 torus
    (1, 3, 50, 32, 8, 1.0),
    (1, 2, 2600, 64, 5, 0.2),    # demes above 1024 members and 256 births: several scan passes
])
def test_space_matches_oracle(X, Y, n0, L, steps, disp):
    c = S.spatial_community(X=X, Y=Y, n0=n0, n_loci=L, mu=1e-3, disp=disp if disp < 1 else 0.999999, seed=3)
    gpu = sp().Space(c, stats_capacity=64)
    orc = oracle.OracleSpace(c)
    gpu.step(steps)
    assert_same(gpu, orc, steps)
    assert gpu.state()["t"] == steps and gpu.state()["status"] == 0


def test_space_graph_chunks_match_oracle():
    """Steps in chunks of 32 replay one captured graph: 70 steps (two chunks
    and 6 direct steps), then a call that replays the cached graph again."""
    c = S.spatial_community(X=3, Y=3, n0=70, n_loci=64, mu=1e-3, disp=0.2, seed=17)
    gpu = sp().Space(c, capacity=60_000, staging_capacity=30_000, stats_capacity=128)  # grows to ~2.1e4
    orc = oracle.OracleSpace(c)
    gpu.step(70)
    assert_same(gpu, orc, 70)
    gpu.step(32)
    assert_same(gpu, orc, 32)
    assert gpu.state()["t"] == 102 and gpu.state()["status"] == 0


def test_space_founders_match_and_stepwise_calls():
    c = S.spatial_community(X=5, Y=4, n0=90, n_loci=128, mu=1e-2, seed=9)
    gpu = sp().Space(c, stats_capacity=32)
    orc = oracle.OracleSpace(c)
    for s in range(3):
        for p in range(20):
            rg, ag = gpu.deme(s, p)
            ro, ao = orc.deme(s, p)
            assert np.array_equal(rg, ro) and np.array_equal(ag, ao)
    for k in (1, 2, 3):
        gpu.step(k)
        assert_same(gpu, orc, k)


def test_space_capacity_overflow_is_reported():
    c = S.spatial_community(X=2, Y=2, n0=100, n_loci=32, seed=1)
    for spc in c.species:
        spc.beta_q16 = 8 * 65536
        spc.bmax = 10_000
        spc.G, spc.E, spc.C = 1000, 0, [0, 0, 0]
    gpu = sp().Space(c, capacity=1500)
    gpu.step(5)
    st = gpu.state()
    assert st["status"] == sp().ERR_RANGE and st["t"] < 5
    assert gpu.sizes().sum() <= 1500


def _popcount(words: np.ndarray) -> int:
    return int(np.unpackbits(np.ascontiguousarray(words).view(np.uint8)).sum())


def test_space_full_size_counts_and_newborns():
    """The measured community (64 x 64 torus, 3 species, 814 founders per
    species and patch, L = 256) after three steps, checked on every deme
    against properties that hold at any size: counts are conserved from step
    to step, every deme stores adults first, and the last step's newborns --
    exactly the age-0 individuals -- agree with its birth, adult,
    heterozygosity and allele-count statistics."""
    c = S.spatial_community()
    g = sp().Space(c, stats_capacity=16)
    g.step(3)
    state = g.state()
    assert state["status"] == 0 and state["t"] == 3
    st = g.read_stats(1, 3)
    assert np.array_equal(st["n_after"], st["survivors"] + st["births"])
    assert np.array_equal(st["n_before"][1:], st["n_after"][:-1])
    sizes = g.sizes()
    assert np.array_equal(sizes.sum(axis=1), st["n_after"][-1])
    assert sizes.sum() == state["total"]
    W = c.n_loci // 32
    for s in range(g.ns):
        young = het = allele = adults = 0
        for p in range(c.patches):
            rec, age = g.deme(s, p)
            assert len(age) == sizes[s, p]
            assert np.all(np.diff(age.astype(np.int64)) <= 0), (s, p)
            new = rec[age == 0]
            young += len(new)
            adults += int((age == 2).sum())
            het += _popcount(new[:, :W] ^ new[:, W:])
            allele += _popcount(new)
        last = st[-1][s]
        assert young == last["births"], s
        assert adults == last["adults_after"], s
        assert het == last["het_newborn"], s
        assert allele == last["allele_newborn"], s
    g.close()
