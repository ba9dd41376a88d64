"""The allocation-free generation call (spg_generation_noalloc) against the
population API, through the C ABI.

Callers that may not allocate device memory -- code running while a stream is
being captured into a CUDA graph, applications whose device memory belongs to
another framework's pool, loops that forbid allocation after start-up -- use
spg_generation_noalloc with their own buffers; its working memory is a fixed
array inside the library.  Two calls in a row must reproduce, bit for bit,
the first two generations that spg_step_generations forms for the same
population (the tolerance the parity tests use for integer outputs)."""
import numpy as np
import pytest

import spegg_synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09255_gb300 import build
    build.build()


def _u32_to_device(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32).copy()).cuda()


def _device_to_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,n_loci", [(50_000, 128), (3_001, 32), (20_000, 256)])
def test_two_allocation_free_generations_match_population_api(n, n_loci):
    from paper_1603_09255_gb300 import spegg as sp
    w = S.single_species(n=n, n_loci=n_loci, mu=1e-3, s=1.5, seed=5, replicate=2)
    w.init_genotypes = S.genotypes_bernoulli(n, n_loci, 0.4, seed=6)
    ref = sp.Population.from_workload(w, stats_capacity=4)
    ref.step(1)
    g1, s1, st1 = ref.genotypes(), ref.survivors(), ref.read_stats(1, 1)
    ref.step(1)
    g2, s2, st2 = ref.genotypes(), ref.survivors(), ref.read_stats(2, 1)

    stream = torch.cuda.current_stream()
    effects = np.ascontiguousarray(w.effects, dtype=np.int16)
    table = np.ascontiguousarray(w.surv_table, dtype=np.uint32)
    parents = _u32_to_device(w.init_genotypes.reshape(-1))
    survivors = torch.arange(n, dtype=torch.int32, device="cuda")
    S_prev = n
    for gen, (g_ref, s_ref, st_ref) in ((1, (g1, s1, st1)), (2, (g2, s2, st2))):
        children = torch.empty_like(parents)
        surv_out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        stats = torch.zeros(sp.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        args = sp.spg_noalloc_generation(
            n, n_loci, w.seed, w.replicate, gen, S_prev, sp.CERTAIN, effects.ctypes.data, table.ctypes.data,
            w.bias, w.shift, w.mu, parents.data_ptr(), survivors.data_ptr(), children.data_ptr(),
            surv_out.data_ptr(), stats.data_ptr())
        sp.generation_noalloc(args, stream.cuda_stream)
        torch.cuda.synchronize()
        st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=sp.STATS_DTYPE)
        assert st.tobytes() == st_ref.tobytes(), f"statistics of generation {gen}"
        assert np.array_equal(_device_to_u32(children).reshape(n, -1), g_ref), f"genotypes of generation {gen}"
        k = int(st[0]["s"])
        assert np.array_equal(_device_to_u32(surv_out)[:k], s_ref), f"survivors of generation {gen}"
        parents, survivors, S_prev = children, surv_out, k


def test_allocation_free_call_rejects_populations_above_its_limit():
    from paper_1603_09255_gb300 import spegg as sp
    e = np.zeros(32, np.int16)
    t = S.constant_table(S.CERTAIN)
    big = 4194304 + 1
    args = sp.spg_noalloc_generation(big, 32, 0, 0, 1, 1, sp.CERTAIN, e.ctypes.data, t.ctypes.data, 0, 0, 0.0,
                                     8, 8, 8, 8, 8)
    with pytest.raises(sp.SpeggError) as err:
        sp.generation_noalloc(args, 0)
    assert err.value.code == sp.ERR_INVALID and "4194304" in str(err.value)
