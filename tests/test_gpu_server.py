"""Served jobs (spg_server_*): continuous batching admits jobs by device
footprint as they arrive, runs resident jobs together in shared launches, and
every job's results equal the same population run alone, bit for bit."""
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


def sp():
    from paper_1603_09255_gb300 import spegg
    return spegg


def small_trace(count=12, seed=5):
    ws, gens, arrivals = S.served_trace(count=count, rate=400.0, n_min=300, n_max=30_000, gen_min=10,
                                        gen_max=70, mu=1e-3, s_max=2.0, trace_seed=seed)
    for i, w in enumerate(ws):
        if i % 4 == 1:  # some jobs carry a logistic resource
            eco = S.consumer_resource(n=w.n, n_loci=w.n_loci, K=8.0 * w.n, seed=w.seed, replicate=w.replicate,
                                      effects_seed=5000 + i)
            ws[i] = eco
            ws[i].mu, ws[i].s = w.mu, w.s
    return ws, gens, arrivals


def alone(w, n_gen):
    p = sp().Population.from_workload(w, stats_capacity=n_gen + 1)
    p.step(n_gen)
    st = p.state()
    out = p.read_stats(1, st["gen"]) if st["gen"] else np.zeros(0, sp().STATS_DTYPE)
    p.close()
    return out, st


def test_served_jobs_equal_jobs_run_alone():
    ws, gens, arrivals = small_trace()
    # a budget that holds only a few jobs at once forces queueing
    srv = sp().Server(memory_budget=48 << 20, max_resident=4, gens_per_tick=8)
    jobs = srv.run_trace(ws, gens, arrivals)
    c = srv.counters()
    assert c["submitted"] == len(ws) and c["queued"] == 0 and c["resident"] == 0
    assert c["peak_memory_used"] <= c["memory_budget"] and c["peak_resident"] <= 4
    admits = []
    for i, (w, g) in enumerate(zip(ws, gens)):
        info = srv.job_info(int(jobs[i]))
        assert info["state"] == 2 and info["t_finish"] >= info["t_admit"] >= info["t_arrival"] - 1e-9
        admits.append(info["t_admit"])
        ref, st = alone(w, g)
        assert info["gen"] == st["gen"] and info["status"] == st["status"]
        got = srv.job_stats(int(jobs[i]), 1, info["gen"]) if info["gen"] else ref
        assert got.tobytes() == ref.tobytes(), f"job {i} differs from the same population run alone"
    assert all(b >= a for a, b in zip(admits, admits[1:])), "admission follows arrival order"
    srv.close()


def test_tick_api_and_states():
    ws, gens, _ = small_trace(5, seed=9)
    srv = sp().Server(max_resident=2, gens_per_tick=16)
    ids = [srv.submit(w, g) for w, g in zip(ws, gens)]
    assert all(srv.job_info(i)["state"] == 0 for i in ids)
    r, q = srv.tick()
    assert r == 2 and q == 3
    assert [srv.job_info(i)["state"] for i in ids[:2]] == [1, 1]
    srv.drain()
    for i, (w, g) in zip(ids, zip(ws, gens)):
        info = srv.job_info(i)
        assert info["state"] == 2
        ref, _ = alone(w, g)
        assert srv.job_stats(i, 1, info["gen"]).tobytes() == ref.tobytes()
    srv.close()


def test_oversized_job_is_rejected():
    srv = sp().Server(memory_budget=1 << 20)
    w = S.single_species(n=200_000, n_loci=256)
    with pytest.raises(sp().SpeggError) as e:
        srv.submit(w, 100)
    assert e.value.code == sp().ERR_BUDGET
    srv.close()


def test_measured_trace_jobs_equal_jobs_run_alone():
    """The measured served trace (48 jobs from a Poisson stream at 200 jobs/s,
    N log-uniform [1e3, 2e6], L in {64, 256}, 100-2000 generations), served
    as the benchmark serves it; a seeded sample of jobs, each re-run alone on
    the GPU, bit for bit."""
    ws, gens, arrivals = S.served_trace(count=48, rate=200.0)
    srv = sp().Server(gens_per_tick=16)
    jobs = srv.run_trace(ws, gens, arrivals)
    assert srv.counters()["queued"] == 0
    rng = np.random.default_rng(11)
    for i in sorted(int(x) for x in rng.choice(len(ws), 6, replace=False)):
        info = srv.job_info(int(jobs[i]))
        ref, st = alone(ws[i], gens[i])
        assert info["state"] == 2 and info["gen"] == st["gen"] and info["status"] == st["status"]
        got = srv.job_stats(int(jobs[i]), 1, info["gen"]) if info["gen"] else ref
        assert got.tobytes() == ref.tobytes(), f"job {i} differs from the same population run alone"
    srv.close()


def test_served_variant_jobs_equal_jobs_run_alone():
    """Jobs with a linkage map, parent weights or both are served beside plain
    jobs and equal the same populations run alone."""
    ws, gens, arrivals = small_trace(count=12, seed=9)
    for i, w in enumerate(ws):
        if i % 4 in (1, 3):
            w = S.with_linkage(w, 2, 1.0)
        if i % 4 in (2, 3):
            w = S.with_weights(w, slope=1.25)
        ws[i] = w
    srv = sp().Server(memory_budget=64 << 20, max_resident=5, gens_per_tick=8)
    jobs = srv.run_trace(ws, gens, arrivals)
    for i, (w, g) in enumerate(zip(ws, gens)):
        info = srv.job_info(int(jobs[i]))
        ref, st = alone(w, g)
        assert info["state"] == 2 and info["gen"] == st["gen"] and info["status"] == st["status"]
        got = srv.job_stats(int(jobs[i]), 1, info["gen"]) if info["gen"] else ref
        assert got.tobytes() == ref.tobytes(), f"job {i} differs from the same population run alone"
    srv.close()


def test_served_continuous_jobs_equal_jobs_run_alone():
    ws, gens, arrivals = small_trace(count=10, seed=13)
    for i, w in enumerate(ws):
        if i % 2 == 0:  # continuous-allele jobs of the same size and locus count
            ws[i] = S.continuous_trait(n=w.n, n_loci=w.n_loci, mu=1e-2, mut_sd=0.1, env_sd=0.1 * (i % 3),
                                       seed=w.seed, replicate=w.replicate, effects_seed=900 + i)
    srv = sp().Server(memory_budget=64 << 20, max_resident=4, gens_per_tick=8)
    jobs = srv.run_trace(ws, gens, arrivals)
    for i, (w, g) in enumerate(zip(ws, gens)):
        info = srv.job_info(int(jobs[i]))
        ref, st = alone(w, g)
        assert info["state"] == 2 and info["gen"] == st["gen"] and info["status"] == st["status"]
        got = srv.job_stats(int(jobs[i]), 1, info["gen"]) if info["gen"] else ref
        assert got.tobytes() == ref.tobytes(), f"job {i} differs from the same population run alone"
    srv.close()
