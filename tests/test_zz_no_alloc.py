"""The allocation-free generation call (spg_generation_noalloc), through the
C ABI, against the population API and the CPU oracle.

Some callers may not allocate device memory: applications whose device
memory belongs entirely to another framework's pool (their own cudaMalloc
would fail or fragment it), plug-ins running inside such a framework under a
fixed budget, and real-time loops that forbid allocation after start-up
because an allocation can block the device or fail at any moment.  They call
spg_generation_noalloc with their own input and output buffers; its working
memory is a fixed array inside the library.  Two calls in a row must
reproduce, bit for bit, the first two generations that spg_step_generations
and the oracle form for the same population (integer outputs: the exact
tolerance every parity test uses).  The array keeps the previous call's
contents, so a call of another shape in between must not change the result.
"""
import numpy as np
import pytest

import oracle
import spegg_synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# statistics fields that depend on the ecology, which the allocation-free call
# does not run (it takes the survival factor as given and reports R = 0)
ECOLOGY_FIELDS = ("consumption", "R", "f")


@pytest.fixture(scope="module", autouse=True)
def gpu_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09255_gb300 import build
    build.build()


def _sp():
    from paper_1603_09255_gb300 import spegg
    return spegg


def _u32_to_device(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32).copy()).cuda()


def _device_to_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def _noalloc_generation(w, gen, S_prev, f, parents, survivors, stream):
    """One allocation-free generation of workload w: (children, survivors,
    statistics record) read back to the host after the stream completes."""
    sp = _sp()
    n = w.n
    effects = np.ascontiguousarray(w.effects, dtype=np.int16)
    table = np.ascontiguousarray(w.surv_table, dtype=np.uint32)
    children = torch.empty_like(parents)
    surv_out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    stats = torch.zeros(sp.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    args = sp.spg_noalloc_generation(
        n, w.n_loci, w.seed, w.replicate, gen, S_prev, f, effects.ctypes.data, table.ctypes.data,
        w.bias, w.shift, w.mu, parents.data_ptr(), survivors.data_ptr(), children.data_ptr(),
        surv_out.data_ptr(), stats.data_ptr())
    sp.generation_noalloc(args, stream)
    torch.cuda.synchronize()
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=sp.STATS_DTYPE)
    return children, surv_out, st


def _assert_generation(children, surv_out, st, n, ref_geno, ref_surv, ref_stats, what, skip=()):
    names = [k for k in ref_stats.dtype.names if k not in skip]
    got = {k: st[0][k] for k in names}
    want = {k: ref_stats[0][k] for k in names}
    assert got == want, f"statistics of {what}"
    assert np.array_equal(_device_to_u32(children).reshape(n, -1), ref_geno), f"genotypes of {what}"
    k = int(st[0]["s"])
    assert np.array_equal(_device_to_u32(surv_out)[:k], ref_surv), f"survivors of {what}"


def _workload(n, n_loci, seed=5, replicate=2):
    w = S.single_species(n=n, n_loci=n_loci, mu=1e-3, s=1.5, seed=seed, replicate=replicate)
    w.init_genotypes = S.genotypes_bernoulli(n, n_loci, 0.4, seed=seed + 1)
    return w


@pytest.mark.parametrize("n,n_loci,legacy_stream", [(50_000, 128, False), (3_001, 32, True), (20_000, 256, False)])
def test_two_allocation_free_generations_match_population_api_and_oracle(n, n_loci, legacy_stream):
    sp = _sp()
    w = _workload(n, n_loci)
    ref = sp.Population.from_workload(w, stats_capacity=4)
    orc = oracle.OraclePopulation.from_workload(w)
    expect = []
    for gen in (1, 2):
        ref.step(1)
        so = orc.step(1)
        g, s, st = ref.genotypes(), ref.survivors(), ref.read_stats(gen, 1)
        # the population API is itself oracle-pinned; both must agree here too
        assert st.tobytes() == so.tobytes() and np.array_equal(g, orc.genotypes())
        assert np.array_equal(s, orc.survivors())
        expect.append((g, s, st))
    ref.close()
    orc.close()

    stream = 0 if legacy_stream else torch.cuda.current_stream().cuda_stream
    parents = _u32_to_device(w.init_genotypes.reshape(-1))
    survivors = torch.arange(n, dtype=torch.int32, device="cuda")
    S_prev = n
    for gen, (g_ref, s_ref, st_ref) in zip((1, 2), expect):
        children, surv_out, st = _noalloc_generation(w, gen, S_prev, sp.CERTAIN, parents, survivors, stream)
        _assert_generation(children, surv_out, st, n, g_ref, s_ref, st_ref, f"generation {gen}")
        parents, survivors, S_prev = children, surv_out, int(st[0]["s"])


def test_allocation_free_generations_with_a_survival_factor_match_oracle():
    """A survival factor below certainty (the resource factor of a
    consumer-resource population, passed in by the caller) scales every
    threshold exactly as the oracle's ecology does."""
    sp = _sp()
    n, n_loci = 30_000, 64
    w = S.consumer_resource(n=n, n_loci=n_loci, mu=1e-3, s=0.5, K=2.0 * n, seed=9, replicate=1)
    w.init_genotypes = S.genotypes_bernoulli(n, n_loci, 0.5, seed=10)
    orc = oracle.OraclePopulation.from_workload(w)
    f_used = [orc.state()["f"]]
    expect = []
    for gen in (1, 2):
        so = orc.step(1)
        expect.append((orc.genotypes(), orc.survivors(), so))
        f_used.append(orc.state()["f"])
    orc.close()
    assert f_used[0] < sp.CERTAIN and f_used[1] < sp.CERTAIN and f_used[0] != f_used[1]

    stream = torch.cuda.current_stream().cuda_stream
    parents = _u32_to_device(w.init_genotypes.reshape(-1))
    survivors = torch.arange(n, dtype=torch.int32, device="cuda")
    S_prev = n
    for gen, (g_ref, s_ref, st_ref) in zip((1, 2), expect):
        children, surv_out, st = _noalloc_generation(w, gen, S_prev, f_used[gen - 1], parents, survivors, stream)
        _assert_generation(children, surv_out, st, n, g_ref, s_ref, st_ref, f"generation {gen}",
                           skip=ECOLOGY_FIELDS)
        assert int(st[0]["f"]) == f_used[gen - 1] and float(st[0]["R"]) == 0.0
        parents, survivors, S_prev = children, surv_out, int(st[0]["s"])


def test_call_of_another_shape_in_between_leaves_no_trace():
    """The fixed array keeps the last call's bitmap, bucket counts, state and
    accumulators; a larger population with another locus count run between
    two generations of the first must not change the second one."""
    sp = _sp()
    w = _workload(40_000, 64, seed=21, replicate=3)
    other = _workload(90_000, 32, seed=31, replicate=4)
    other.surv_table = S.constant_table(0x40000000)  # about a quarter survive: other bucket counts
    orc = oracle.OraclePopulation.from_workload(w)
    expect = []
    for _ in (1, 2):
        so = orc.step(1)
        expect.append((orc.genotypes(), orc.survivors(), so))
    orc.close()

    stream = torch.cuda.current_stream().cuda_stream
    parents = _u32_to_device(w.init_genotypes.reshape(-1))
    survivors = torch.arange(w.n, dtype=torch.int32, device="cuda")
    c1, s1, st1 = _noalloc_generation(w, 1, w.n, sp.CERTAIN, parents, survivors, stream)
    _assert_generation(c1, s1, st1, w.n, *expect[0], "generation 1")
    o_par = _u32_to_device(other.init_genotypes.reshape(-1))
    o_surv = torch.arange(other.n, dtype=torch.int32, device="cuda")
    _, _, ost = _noalloc_generation(other, 5, other.n, sp.CERTAIN, o_par, o_surv, stream)
    assert 0 < int(ost[0]["s"]) < other.n // 2
    c2, s2, st2 = _noalloc_generation(w, 2, int(st1[0]["s"]), sp.CERTAIN, c1, s1, stream)
    _assert_generation(c2, s2, st2, w.n, *expect[1], "generation 2 after another call")


def test_allocation_free_call_rejects_populations_above_its_limit():
    sp = _sp()
    e = np.zeros(32, np.int16)
    t = S.constant_table(S.CERTAIN)
    big = 4194304 + 1
    args = sp.spg_noalloc_generation(big, 32, 0, 0, 1, 1, sp.CERTAIN, e.ctypes.data, t.ctypes.data, 0, 0, 0.0,
                                     8, 8, 8, 8, 8)
    with pytest.raises(sp.SpeggError) as err:
        sp.generation_noalloc(args, 0)
    assert err.value.code == sp.ERR_INVALID and "4194304" in str(err.value)
