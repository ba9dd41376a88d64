"""Benchmark of the per-generation update on one GB300.

A step is one pass of the hot path over the consumer-resource workload:
N = 1,000,000 diploid individuals, L = 128 loci (4 words per haplotype),
mu = 1e-5, Gaussian stabilising viability (s = 0.5), logistic resource
(r = 0.5, K = 1e7, R0 = K/2, R_half = K/10), 1,000 generations.  The metric is
individual-generations per second (N x generations / time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (test infrastructure, single thread) on a
bounded sample of the same workload.  Under torchrun (N > 1) every rank runs an
independent replica of the workload (replicas only, no collective on the data
path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import spegg_synth as S  # noqa: E402

GENERATIONS = 1000
# Algorithmic bytes per offspring-generation: two survivor-index reads (8 B),
# two parent records (2 x 8W B), the child record (8W B), one survivor index
# write (4 B) = 12 + 24W.
def algorithmic_bytes(words: int) -> int:
    return 12 + 24 * words


# DRAM traffic per launch of the dominant kernel from one ncu capture, keyed by
# the hash of the kernel source it was taken on (null once the kernel changes).
MEASURED_TRAFFIC = {"84b7b55419a84a47": 36823296}


def kernel_source_hash() -> str:
    with open(os.path.join(ROOT, "paper_1603_09255_gb300", "csrc", "kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"spegg_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [x for x in sm if smax and x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def replica_workload(workload, rank: int):
    """Replicas only: rank r runs the same population with replicate id r
    (independent Philox streams, no exchange between ranks)."""
    workload.replicate = rank
    return workload


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (timings: the slowest rank sets the
    whole job's time); the value itself without an initialised group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reference_arm(args, workload):
    """The CPU oracle timed on a bounded sample: each step is one generation of
    the full-size population, single-threaded."""
    import oracle
    rank, _, ws = dist_env()
    if rank != 0:
        return
    pop = oracle.OraclePopulation.from_workload(workload)
    for _ in range(args.warmup):
        pop.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pop.step(1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = workload.n * args.steps / total
    sample = f"{args.steps} generation(s) of the N={workload.n}, L={workload.n_loci} population after {args.warmup} warm-up"
    line = {
        "impl": "reference", "metric": "individual-generations/s", "value": value,
        "unit": "individual-generations/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": bench_config(workload, "none (CPU)"),
        "cpu_baseline": {"value": value, "unit": "individual-generations/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "individual-generations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def bench_config(w, l2):
    return {"workload": f"consumer-resource N={w.n} L={w.n_loci} mu={w.mu:g} s={w.s} r={w.eco_r} K={w.eco_K:g}, "
                        f"{GENERATIONS} generations per step",
            "n": w.n, "n_loci": w.n_loci, "generations_per_step": GENERATIONS, "l2": l2}


def batched_replicates(spegg, torch, gens: int = 500, plain_members: int = 256, plain_gens: int = 32,
                       oracle_cpu: bool = False, count: int = 4096):
    """Batched-replicates workload: 4,096 independent single-species runs (N
    log-uniform in [1e3, 2e5], L in {32, 64, 128}, s in [0, 0.5]) advanced by
    shared, graph-captured launches with autotuned tilings, against the plain
    path (one population at a time) timed on the first `plain_members`."""
    ws = S.batch_replicates(count=count, n_gen=gens)
    plain_members = min(plain_members, count)
    stream = torch.cuda.Stream()
    batch = spegg.Batch(ws, stats_capacity=gens + 64, stream=stream)
    ran = batch.autotune(4)
    batch.step(32)
    batch.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
    batch.step(gens)
    with torch.cuda.stream(stream):
        b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b)
    sum_n = sum(w.n for w in ws)
    tilings = {str(L): batch.launch_shape(L) for L in (32, 64, 128)}
    tuned = getattr(batch, "autotune_report", {})
    # per-generation latency of the whole batch: single generations bracketed
    # by events, after 3 untimed ones
    batch.step(3)
    g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(32)]
    for ga, gb in g_ev:
        with torch.cuda.stream(stream):
            ga.record(stream)
        batch.step(1)
        with torch.cuda.stream(stream):
            gb.record(stream)
    stream.synchronize()
    gen_ms = [ga.elapsed_time(gb) for ga, gb in g_ev]
    batch.close()
    pops = [spegg.Population.from_workload(ws[i], stats_capacity=64, stream=stream) for i in range(plain_members)]
    for p in pops:
        p.step(1)
    stream.synchronize()
    with torch.cuda.stream(stream):
        a.record(stream)
    for p in pops:
        p.step(plain_gens)
    with torch.cuda.stream(stream):
        b.record(stream)
    stream.synchronize()
    ms_plain = a.elapsed_time(b)
    plain = sum(ws[i].n for i in range(plain_members)) * plain_gens / (ms_plain / 1e3)
    for p in pops:
        p.close()
    value = sum_n * gens / (ms / 1e3)
    # algorithmic bytes of one generation of every replicate: sum of N (12 + 24W)
    algo = sum(w.n * algorithmic_bytes(w.words) for w in ws) * gens
    peak, source = load_peaks()
    achieved = algo / (ms / 1e3) / 1e9
    return {"workload": f"4096 replicates, N log-uniform [1e3, 2e5] (sum {sum_n}), L in {{32, 64, 128}}, "
                        f"s in [0, 0.5], {gens} generations timed after {ran + 32}",
            "value": value, "unit": "individual-generations/s", "ms": ms, "tilings": tilings, "autotune": tuned,
            "plain_value": plain, "plain_sample": f"first {plain_members} replicates, {plain_gens} generations, "
                                                  "one population stepped at a time",
            "speedup_vs_plain": value / plain,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "note": f"sum of N (12 + 24W) B per generation, of {source}"},
            "per_generation": {"p50_ms": float(np.percentile(gen_ms, 50)), "p99_ms": float(np.percentile(gen_ms, 99)),
                               "repeats": len(gen_ms), "warmup": 3},
            "cpu_baseline": oracle_batched_baseline(ws) if oracle_cpu else None}


def served_sweep(spegg, torch, count: int = 48, rate: float = 200.0):
    """Served parameter sweep: a seeded Poisson stream (rate jobs/s) of jobs
    with N log-uniform in [1e3, 2e6], L in {64, 256}, 100-2000 generations,
    admitted by device footprint and run by continuous batching; latency is
    arrival -> finish on the server's clock."""
    ws, gens, arrivals = S.served_trace(count=count, rate=rate)
    srv = spegg.Server(gens_per_tick=16)
    t0 = time.perf_counter()
    jobs = srv.run_trace(ws, gens, arrivals)
    wall = time.perf_counter() - t0
    infos = [srv.job_info(int(j)) for j in jobs]
    lat = np.array([i["t_finish"] - i["t_arrival"] for i in infos])
    work = sum(w.n * i["gen"] for w, i in zip(ws, infos))
    makespan = max(i["t_finish"] for i in infos) - min(i["t_arrival"] for i in infos)
    c = srv.counters()
    srv.close()
    value = work / makespan
    mean_job = work / count
    return {"workload": f"{count} jobs, Poisson {rate:g}/s, N log-uniform [1e3, 2e6], L in {{64, 256}}, "
                        "100-2000 generations, continuous batching",
            "value": value, "unit": "individual-generations/s", "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "makespan_s": makespan, "wall_s": wall,
            "offered_load": rate * mean_job / value, "peak_resident": c["peak_resident"],
            "peak_memory_gb": c["peak_memory_used"] / 1e9}


def variant_population(spegg, torch, w, label: str, gens: int = 256, bytes_per_offspring=None):
    """One variant of the consumer-resource population (N = 10^6, L = 128),
    `gens` generations after 64, L2 flushed before, CUDA events on its stream."""
    stream = torch.cuda.Stream()
    pop = spegg.Population.from_workload(w, stats_capacity=gens + 128, stream=stream)
    pop.step(64)
    pop.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        flush.fill_(7)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
    pop.step(gens)
    with torch.cuda.stream(stream):
        b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b)
    peak, source = load_peaks()
    per = bytes_per_offspring if bytes_per_offspring is not None else 12 + 24 * w.words
    achieved = w.n * per * gens / (ms / 1e3) / 1e9
    out = {"workload": f"{w.name.split('+')[0]} N={w.n} L={w.n_loci}, {label}, "
                       f"{gens} generations after 64 (L2 flushed before)",
           "value": w.n * gens / (ms / 1e3), "unit": "individual-generations/s", "us_per_generation": ms * 1e3 / gens,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "note": f"{per} B per offspring (algorithmic), of {source}"}}
    pop.close()
    return out


def spatial_community(spegg, torch, steps: int = 200, oracle_cpu: bool = False):
    """Three-species community on a 64 x 64 torus, 814 founders per species
    and patch (1.0e7 individuals), L = 256, age classes 0/1/2, dispersal 0.05,
    200 steps; throughput in individual-steps per second."""
    c = S.spatial_community()
    stream = torch.cuda.Stream()
    g = spegg.Space(c, stream=stream, stats_capacity=steps + 8)
    g.step(3)
    g.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
    g.step(steps)
    with torch.cuda.stream(stream):
        b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b)
    st = g.read_stats(4, steps)
    ind = int(st["n_before"].sum())
    births = int(st["births"].sum())
    words = c.n_loci // 32
    # algorithmic bytes: every member's record (8W B) and age read once and
    # written once at its new place; every newborn reads two parent records
    # and is written once with its age
    algo = ind * (16 * words + 2) + births * (24 * words + 1)
    peak, source = load_peaks()
    achieved = algo / (ms / 1e3) / 1e9
    out = {"workload": f"3 species on a 64 x 64 torus, {c.species[0].n0} founders per species and patch, "
                       f"L={c.n_loci}, dispersal 0.05, {steps} steps after 3",
           "value": ind / (ms / 1e3), "unit": "individual-steps/s", "ms_per_step": ms / steps,
           "individuals_first_step": int(st[0]["n_before"].sum()), "individuals_last_step": int(st[-1]["n_after"].sum()),
           "births": births,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "note": f"whole step (8 launches), of {source}"},
           "cpu_baseline": oracle_spatial_baseline() if oracle_cpu else None}
    g.close()
    return out


def _oracle_generations(job):
    """Pool worker: one workload on the oracle; (individual-generations, seconds
    of its generation steps)."""
    w, gens = job
    import oracle
    pop = oracle.OraclePopulation.from_workload(w)
    t0 = time.perf_counter()
    pop.step(gens)
    return w.n * gens, time.perf_counter() - t0


def oracle_batched_baseline(ws, members: int = 64, gens: int = 2):
    """The oracle on the first `members` replicates, one process per core
    (spawned: safe after CUDA initialisation); the value is the summed
    per-process step rate."""
    import multiprocessing as mp
    sample = ws[:members]
    cores = max(1, min(len(sample), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_generations, [(w, gens) for w in sample], chunksize=1)
    ind = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    return {"value": ind / busy * cores, "unit": "individual-generations/s", "cores": cores, "kind": "oracle",
            "sample": f"first {members} replicates ({sum(w.n for w in sample)} individuals), {gens} generations "
                      f"each, {cores} processes; value = individual-generations / step seconds x processes"}


def oracle_spatial_baseline(X: int = 8, Y: int = 8, steps: int = 4):
    """The oracle on an X x Y torus with the measured community's per-patch
    density, single thread."""
    import oracle
    c = S.spatial_community(X=X, Y=Y)
    sp = oracle.OracleSpace(c)
    sp.step(1)
    t0 = time.perf_counter()
    st = sp.step(steps)
    dt = time.perf_counter() - t0
    ind = int(st["n_before"].sum())
    sp.close()
    return {"value": ind / dt, "unit": "individual-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{X} x {Y} torus, same species and per-patch density ({ind // steps} individuals), "
                      f"{steps} steps after 1, single thread, {dt:.1f} s"}


def cpu_baseline(workload, target_seconds=12.0):
    import oracle
    pop = oracle.OraclePopulation.from_workload(workload)
    t0 = time.perf_counter()
    gens = 0
    while time.perf_counter() - t0 < target_seconds and gens < 20:
        pop.step(1)
        gens += 1
    dt = time.perf_counter() - t0
    return {"value": workload.n * gens / dt, "unit": "individual-generations/s", "cores": 1, "kind": "oracle",
            "sample": f"first {gens} generations of the N={workload.n}, L={workload.n_loci} consumer-resource "
                      f"population, single thread, {dt:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="omit the CPU oracle baseline measurement")
    ap.add_argument("--no-batched", action="store_true", help="omit the batched-replicates measurement")
    ap.add_argument("--no-served", action="store_true", help="omit the served-sweep measurement")
    ap.add_argument("--no-spatial", action="store_true", help="omit the spatial-community measurement")
    ap.add_argument("--no-linked", action="store_true", help="omit the linkage-map measurement")
    ap.add_argument("--no-weighted", action="store_true", help="omit the weighted-parents measurement")
    ap.add_argument("--no-dominance", action="store_true", help="omit the dominance measurement")
    ap.add_argument("--no-continuous", action="store_true", help="omit the continuous-allele measurement")
    ap.add_argument("--shape", default="", metavar="B,I",
                    help="launch shape of the headline population: threads per block, offspring per thread; "
                         "results do not depend on it")
    ap.add_argument("--only-batched", type=int, default=0, metavar="R",
                    help="run only the batched-replicates measurement on the first R replicates (profiling)")
    args = ap.parse_args()
    workload = S.consumer_resource()
    if args.only_batched:
        import torch
        from paper_1603_09255_gb300 import build as pkg_build
        pkg_build.build()
        from paper_1603_09255_gb300 import spegg
        print(json.dumps(batched_replicates(spegg, torch, gens=args.steps, count=args.only_batched)))
        return
    if args.impl == "reference":
        reference_arm(args, workload)
        return

    import torch
    from paper_1603_09255_gb300 import build as pkg_build
    rank, local_rank, ws = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    pkg_build.build()
    from paper_1603_09255_gb300 import spegg

    workload = replica_workload(workload, rank)
    stream = torch.cuda.Stream()
    pop = spegg.Population.from_workload(workload, stats_capacity=GENERATIONS + 8, stream=stream)
    if args.shape:
        pop.set_launch_shape(*[int(x) for x in args.shape.split(",")])
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        pop.step(GENERATIONS)
    pop.synchronize()

    # timed region: K steps, L2 flushed before each, CUDA events on the stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local_rank) as clocks:
        barrier()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
            pop.step(GENERATIONS)
            with torch.cuda.stream(stream):
                ev[i][1].record(stream)
        stream.synchronize()
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, device="cuda")
    st = pop.state()
    assert st["status"] == 0, f"population status {st['status']}"
    ind_gen = workload.n * GENERATIONS * args.steps
    value = ind_gen * ws / (total_ms / 1000.0)

    # each generation is one offspring launch and one compaction launch; the
    # offspring kernel dominates, the pair is timed together
    launches = GENERATIONS * args.steps
    avg_launch_s = total_ms / 1000.0 / launches
    peak, peak_kind = load_peaks()
    bytes_per_launch = algorithmic_bytes(workload.words) * workload.n
    achieved = bytes_per_launch / avg_launch_s / 1e9
    traffic = MEASURED_TRAFFIC.get(kernel_source_hash())

    # kernel-only duration and per-generation latency: single generations
    # (direct launches) bracketed by events, after 3 untimed ones
    pop.step(3)
    k_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
    for a, b in k_ev:
        with torch.cuda.stream(stream):
            a.record(stream)
        pop.step(1)
        with torch.cuda.stream(stream):
            b.record(stream)
    stream.synchronize()
    gen_us = [a.elapsed_time(b) * 1000.0 for a, b in k_ev]
    kernel_ms = statistics.median(gen_us) / 1000.0

    # end to end through the C ABI with host buffers: restore the population
    # from pinned host memory, run the generations, read the statistics back
    blob = pop.checkpoint()
    pinned = torch.empty(len(blob), dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = np.frombuffer(blob, dtype=np.uint8)
    e2e_times = []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pop.restore_from(pinned.data_ptr(), len(blob))
        g0 = pop.state()["gen"]
        pop.step(GENERATIONS)
        stats = pop.read_stats(g0 + 1, GENERATIONS)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = workload.n * GENERATIONS * ws / (sum(e2e_times) / len(e2e_times))
    assert len(stats) == GENERATIONS

    oracle_cpu = rank == 0 and not args.no_cpu_baseline
    batched = None if args.no_batched else batched_replicates(spegg, torch, oracle_cpu=oracle_cpu)
    served = None if args.no_served else served_sweep(spegg, torch)
    spatial = None if args.no_spatial else spatial_community(spegg, torch, oracle_cpu=oracle_cpu)
    linked = None if args.no_linked else variant_population(
        spegg, torch, S.with_linkage(S.consumer_resource(), 4, 1.0), "linkage map 4 chromosomes x 1 Morgan")
    weighted = None if args.no_weighted else variant_population(
        spegg, torch, S.with_weights(S.consumer_resource()), "parents weighted by trait (1 + tanh z; fathers 2z)")
    dominance = None if args.no_dominance else variant_population(
        spegg, torch, S.with_dominance(S.consumer_resource()), "dominance deviations N(0, 0.1) at every locus")
    continuous = None if args.no_continuous else variant_population(
        spegg, torch, S.continuous_trait(n=1_000_000, n_loci=128, mu=1e-3, mut_sd=0.05, env_sd=0.2),
        "continuous allelic values (int16 Q8), mu 1e-3, mutation sd 0.05, environmental sd 0.2, no resource",
        gens=64, bytes_per_offspring=12 + 12 * 128)
    if rank != 0:
        return
    line = {
        "metric": "individual-generations/s", "value": value, "unit": "individual-generations/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "p50_ms_per_step": float(np.percentile(step_ms, 50)), "p99_ms_per_step": float(np.percentile(step_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": bench_config(workload, "flushed before every step (256 MB write)"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": f"k_offspring<W={workload.words}> + k_compact (one generation)",
                     "shape": pop.launch_shape(),
                     "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6,
                     "isolated_launch_us": kernel_ms * 1000.0},
        "e2e": {"value": e2e_value, "unit": "individual-generations/s", "h2d_bytes_per_step": len(blob),
                "d2h_bytes_per_step": int(stats.nbytes)},
        "gpu_launches": 2 * launches,
        "clocks": clocks.summary(),
        "per_generation": {"p50_us": float(np.percentile(gen_us, 50)), "p99_us": float(np.percentile(gen_us, 99)),
                           "repeats": len(gen_us), "warmup": 3,
                           "note": "one generation (two launches, no graph) bracketed by CUDA events"},
    }
    if batched is not None:
        line["batched"] = batched
    if served is not None:
        line["served"] = served
    if spatial is not None:
        line["spatial"] = spatial
    if linked is not None:
        line["linked"] = linked
    if weighted is not None:
        line["weighted"] = weighted
    if dominance is not None:
        line["dominance"] = dominance
    if continuous is not None:
        line["continuous"] = continuous
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(workload)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
