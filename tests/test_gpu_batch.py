"""Batched replicates (spg_batch_*) through the C ABI: every member equals
the same population stepped alone (and, for a sample, the CPU oracle) bit for
bit; the launch-shape autotuner and tilings never change results."""
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


def sp():
    from paper_1603_09255_gb300 import spegg
    return spegg


def mixed_workloads(count=24, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    sizes = [1, 2, 33, 255, 1000, 1025, 4096, 4097, 9001, 30000]
    for r in range(count):
        n = sizes[r % len(sizes)] if r < len(sizes) else int(rng.integers(100, 40000))
        L = [32, 64, 128, 256][r % 4]
        s = float(rng.uniform(0.0, 2.0))
        if r % 5 == 3:
            w = S.consumer_resource(n=n, n_loci=L, mu=1e-3, s=s, K=max(4.0 * n, 100.0), seed=11, replicate=r,
                                    effects_seed=100 + r)
        else:
            w = S.single_species(n=n, n_loci=L, mu=1e-3, s=s, seed=11, replicate=r, effects_seed=100 + r)
        if r % 7 == 2:
            w.surv_table = S.constant_table(0)  # goes extinct in its first generation
        out.append(w)
    return out


def assert_member_equals(batch, i, ref_stats, ref_geno, ref_surv, ref_state):
    st = batch.state(i)
    assert {k: st[k] for k in ("gen", "S", "status", "f", "R")} == \
        {k: ref_state[k] for k in ("gen", "S", "status", "f", "R")}, i
    got = batch.read_stats(i, 1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
    assert got.tobytes() == ref_stats.tobytes(), i
    assert np.array_equal(batch.genotypes(i), ref_geno), i
    assert np.array_equal(batch.survivors(i), ref_surv), i


def test_batch_members_equal_standalone_populations():
    ws = mixed_workloads()
    n_gen = 40  # one cached 32-generation graph and an 8-generation remainder
    b = sp().Batch(ws, stats_capacity=64)
    b.step(n_gen)
    for i, w in enumerate(ws):
        p = sp().Population.from_workload(w, stats_capacity=64)
        p.step(n_gen)
        st = p.state()
        ref = p.read_stats(1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
        assert_member_equals(b, i, ref, p.genotypes(), p.survivors(), st)
        p.close()


@pytest.mark.parametrize("member", [0, 3, 5, 8, 13])
def test_batch_members_equal_oracle(member):
    ws = mixed_workloads()
    b = sp().Batch(ws, stats_capacity=16)
    b.step(6)
    w = ws[member]
    orc = oracle.OraclePopulation.from_workload(w)
    so = orc.step(6)
    st = orc.state()
    assert_member_equals(b, member, so, orc.genotypes(), orc.survivors(), st)


# the candidates the autotuner times (threads per block, offspring per
# thread, lanes per offspring)
NARROW = [(128, 1, 1), (128, 2, 1), (256, 1, 1), (256, 2, 1), (512, 1, 1), (512, 2, 1)]
WIDE = [(128, 1, 1), (256, 1, 1), (512, 1, 1), (128, 1, 2), (256, 1, 2), (512, 1, 2)]


def test_autotune_and_launch_shapes_do_not_change_results():
    ws = mixed_workloads(12, seed=3)
    a = sp().Batch(ws, stats_capacity=128)
    ran = a.autotune(2)
    assert ran == 18  # six shapes, each one untimed and two timed generations
    for L in (32, 64, 128, 256):
        cands = WIDE if L >= 128 else NARROW
        assert a.launch_shape(L) in cands, L
        rep = a.autotune_report[L]
        assert rep["shape"] == a.launch_shape(L) and 0 < rep["best_ms"] <= rep["worst_ms"]
    a.step(30)
    # the same members stepped through every candidate shape in turn
    b = sp().Batch(ws, stats_capacity=128)
    done = 0
    for k in range(6):
        for L in (32, 64, 128, 256):
            b.set_launch_shape(L, *(WIDE if L >= 128 else NARROW)[k])
        b.step(8)
        done += 8
    b.set_tiling(64, 2)
    b.set_tiling(128, 1)
    b.step(ran + 30 - done)
    for i in range(len(ws)):
        st = a.state(i)
        ref = b.read_stats(i, 1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
        assert_member_equals(a, i, ref, b.genotypes(i), b.survivors(i), b.state(i))


def test_batch_rejects_unsupported_launch_shapes():
    b = sp().Batch(mixed_workloads(4), stats_capacity=8)
    for L, shape in ((32, (64, 1, 1)), (64, (256, 4, 1)), (256, (256, 2, 1)), (128, (512, 2, 1)), (64, (256, 1, 2)),
                     (128, (256, 1, 3)), (48, (256, 1, 1))):
        with pytest.raises(sp().SpeggError):
            b.set_launch_shape(L, *shape)
    b.close()


def test_batch_full_size_sampled_members_equal_oracle():
    """The measured batch (4,096 replicates, N log-uniform [1e3, 2e5], L in
    {32, 64, 128}) for three generations; a seeded sample of members, each
    recomputed alone by the oracle, bit for bit."""
    ws = S.batch_replicates(count=4096, n_gen=64)
    b = sp().Batch(ws, stats_capacity=8)
    b.step(3)
    rng = np.random.default_rng(5)
    for i in sorted(int(x) for x in rng.choice(len(ws), 8, replace=False)):
        orc = oracle.OraclePopulation.from_workload(ws[i])
        so = orc.step(3)
        assert_member_equals(b, i, so, orc.genotypes(), orc.survivors(), orc.state())
    b.close()


def variant_workloads():
    """Every (locus count, variant) pair once: plain, linkage map, parent
    weights, both; ragged sizes, some with the logistic resource."""
    out = []
    sizes = [1, 33, 1000, 4097, 9001, 20000, 2049]
    for r in range(16):
        n_loci, kind, n = [32, 64, 128, 256][r % 4], r // 4, sizes[r % len(sizes)]
        if r % 3 == 0:
            w = S.consumer_resource(n=n, n_loci=n_loci, mu=2e-3, s=1.0, K=max(4.0 * n, 100.0), seed=13, replicate=r,
                                    effects_seed=300 + r)
        else:
            w = S.single_species(n=n, n_loci=n_loci, mu=2e-3, s=1.5, seed=13, replicate=r, effects_seed=300 + r)
        if kind & 1:
            w = S.with_linkage(w, [1, 2, 4][r % 3], 0.5 + 0.5 * (r % 3))
        if kind & 2:
            w = S.with_weights(w, slope=1.0 + 0.25 * (r % 3))
        out.append(w)
    return out


def test_batch_variant_members_equal_standalone_populations():
    """Members with a linkage map, parent weights or both share launches with
    plain members and equal the same populations stepped alone."""
    ws = variant_workloads()
    n_gen = 40
    b = sp().Batch(ws, stats_capacity=64)
    b.step(n_gen)
    for i, w in enumerate(ws):
        p = sp().Population.from_workload(w, stats_capacity=64)
        p.step(n_gen)
        st = p.state()
        ref = p.read_stats(1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
        assert_member_equals(b, i, ref, p.genotypes(), p.survivors(), st)
        p.close()
    b.close()


@pytest.mark.parametrize("member", [5, 6, 10, 11, 12, 13, 15])
def test_batch_variant_members_equal_oracle(member):
    ws = variant_workloads()
    b = sp().Batch(ws, stats_capacity=16)
    b.step(5)
    orc = oracle.OraclePopulation.from_workload(ws[member])
    so = orc.step(5)
    assert_member_equals(b, member, so, orc.genotypes(), orc.survivors(), orc.state())
    b.close()


def test_autotune_advances_variant_members_alike():
    ws = variant_workloads()
    b = sp().Batch(ws, stats_capacity=64)
    ran = b.autotune(1)
    b.step(3)
    for i, w in enumerate(ws):
        p = sp().Population.from_workload(w, stats_capacity=64)
        p.step(ran + 3)
        st = p.state()
        ref = p.read_stats(1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
        assert_member_equals(b, i, ref, p.genotypes(), p.survivors(), st)
        p.close()
    b.close()


def continuous_workloads():
    """Continuous-allele members at every locus count (ragged sizes, one with
    the logistic resource, one with caller founders) among plain members."""
    out = []
    sizes = [1, 300, 2500, 4097, 9001]
    for r in range(10):
        n_loci, n = [32, 64, 128, 256][r % 4], sizes[r % len(sizes)]
        if r % 2 == 0:
            w = S.continuous_trait(n=n, n_loci=n_loci, mu=1e-2, mut_sd=0.1, env_sd=0.2 * (r % 3), seed=21,
                                   replicate=r, effects_seed=700 + r)
            if r == 4:
                w = dataclasses.replace(w, eco_r=0.5, eco_K=4.0 * n, eco_R0=2.0 * n, eco_R_half=0.4 * n,
                                        attack=S.attack_table(w.bias, w.shift))
            if r == 6:
                rng = np.random.default_rng(6)
                w = dataclasses.replace(w, init_values=rng.integers(-300, 300, (n, 2 * n_loci)).astype(np.int16))
        else:
            w = S.single_species(n=n, n_loci=n_loci, mu=1e-3, s=1.0, seed=21, replicate=r, effects_seed=700 + r)
        out.append(w)
    return out


def test_batch_continuous_members_equal_oracle():
    """Continuous-allele members share launches (one block per 256 offspring,
    the block's member from the launch's tile map) and equal the oracle."""
    ws = continuous_workloads()
    b = sp().Batch(ws, stats_capacity=16)
    b.step(6)
    for i, w in enumerate(ws):
        orc = oracle.OraclePopulation.from_workload(w)
        so = orc.step(6)
        st = b.state(i)
        assert {k: st[k] for k in ("gen", "S", "status", "f", "R")} == \
            {k: orc.state()[k] for k in ("gen", "S", "status", "f", "R")}, i
        got = b.read_stats(i, 1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
        assert got.tobytes() == so.tobytes(), i
        assert np.array_equal(b.survivors(i), orc.survivors()), i
        if int(getattr(w, "allele_model", 0)) == 1:
            assert np.array_equal(b.values(i), orc.values()), i
        else:
            assert np.array_equal(b.genotypes(i), orc.genotypes()), i
    b.close()


def test_batch_continuous_members_equal_standalone_over_a_graph():
    ws = continuous_workloads()
    b = sp().Batch(ws, stats_capacity=64)
    ran = b.autotune(1) + 40
    b.step(40)
    for i, w in enumerate(ws):
        p = sp().Population.from_workload(w, stats_capacity=64)
        p.step(ran)
        st = p.state()
        ref = p.read_stats(1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
        assert_member_equals(b, i, ref, p.genotypes(), p.survivors(), st)
        p.close()
    b.close()
