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


def set_generations(g: int) -> None:
    global GENERATIONS
    GENERATIONS = max(1, int(g))
# Algorithmic bytes per offspring-generation: two survivor-index reads (8 B),
# two parent records (2 x 8W B), the child record (8W B), one survivor index
# write (4 B) = 12 + 24W.
def algorithmic_bytes(words: int) -> int:
    return 12 + 24 * words


# DRAM traffic per launch of the dominant kernel (the offspring kernel of the
# headline population) from one ncu capture, keyed by the hash of that
# kernel's sources (null once they change).
MEASURED_TRAFFIC = {"e961a201f358e511": 28457472}
TRAFFIC_SOURCES = ("offspring.cuh", "device_common.cuh", "offspring_w4.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1603_09255_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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
    return {"workload": "consumer-resource", "n": w.n, "n_loci": w.n_loci, "generations_per_step": GENERATIONS,
            "l2": l2}


def timed_on(stream, torch, fn):
    """Milliseconds of fn() on `stream`, CUDA events on the stream."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
    fn()
    with torch.cuda.stream(stream):
        b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b)


def per_generation_ms(stream, torch, step_one, repeats=32, warmup=3):
    """p50/p99 of single generations (direct launches) bracketed by events."""
    for _ in range(warmup):
        step_one()
    stream.synchronize()
    t = [timed_on(stream, torch, step_one) for _ in range(repeats)]
    return float(np.percentile(t, 50)), float(np.percentile(t, 99))


def single_species(spegg, torch, oracle_cpu: bool):
    """The single-species workload (N = 10^4, L = 32, 100 generations): through
    the cached graph (one step call), by direct launches (100 single-generation
    calls), and the oracle single-threaded on the full run.  Each timed run
    starts from the founders restored from a checkpoint, after one untimed run
    of the same calls (which builds the cached graph)."""
    w = S.single_species()
    stream = torch.cuda.Stream()
    ind = w.n * w.n_gen
    times = {}
    for mode in ("graph", "direct"):
        ms = []
        for _ in range(4):  # the first of four runs is a warm-up
            pop = spegg.Population.from_workload(w, stats_capacity=w.n_gen + 8, stream=stream)
            founders = pop.checkpoint()
            if mode == "graph":
                run = lambda: pop.step(w.n_gen)  # noqa: E731
            else:
                run = lambda: [pop.step(1) for _ in range(w.n_gen)]  # noqa: E731
            run()
            pop.restore(founders)
            pop.synchronize()
            ms.append(timed_on(stream, torch, run))
            pop.close()
        times[mode] = min(ms[1:])
    out = {"value": ind / (times["graph"] / 1e3), "nograph": ind / (times["direct"] / 1e3)}
    if oracle_cpu:
        import oracle
        orc = oracle.OraclePopulation.from_workload(w)
        t0 = time.perf_counter()
        orc.step(w.n_gen)
        out["cpu"] = ind / (time.perf_counter() - t0)
        orc.close()
    return out


def batched_replicates(spegg, torch, gens: int = 500, plain_members: int = 0, plain_gens: int = 32,
                       oracle_cpu: bool = False, count: int = 4096):
    """Batched-replicates workload: `count` independent single-species runs (N
    log-uniform in [1e3, 2e5], L in {32, 64, 128}, s in [0, 0.5]) advanced by
    shared, graph-captured launches with autotuned launch shapes, against the
    plain path: every replicate (or the first `plain_members`) stepped one
    population at a time through its own cached graph, 256 populations resident
    at a time, each graph built before its timed run (as the batch's are)."""
    ws = S.batch_replicates(count=count, n_gen=gens)
    plain_members = min(plain_members or count, count)
    stream = torch.cuda.Stream()
    batch = spegg.Batch(ws, stats_capacity=gens + 64, stream=stream)
    batch.autotune(4)
    batch.step(32)
    batch.synchronize()
    ms = timed_on(stream, torch, lambda: batch.step(gens))
    sum_n = sum(w.n for w in ws)
    tuned = getattr(batch, "autotune_report", {})
    p50, p99 = per_generation_ms(stream, torch, lambda: batch.step(1))
    batch.close()
    ms_plain, plain_work = 0.0, 0
    for c0 in range(0, plain_members, 256):
        idx = range(c0, min(c0 + 256, plain_members))
        pops = [spegg.Population.from_workload(ws[i], stats_capacity=2 * plain_gens + 8, stream=stream) for i in idx]
        for p in pops:
            p.step(plain_gens)  # builds each population's cached graph
        stream.synchronize()
        ms_plain += timed_on(stream, torch, lambda: [p.step(plain_gens) for p in pops])
        plain_work += sum(ws[i].n for i in idx) * plain_gens
        for p in pops:
            p.close()
    plain = plain_work / (ms_plain / 1e3)
    value = sum_n * gens / (ms / 1e3)
    # algorithmic bytes of one generation of every replicate: sum of N (12 + 24W)
    algo = sum(w.n * algorithmic_bytes(w.words) for w in ws) * gens
    peak, _ = load_peaks()
    out = {"value": value, "vs_plain": value / plain, "frac": algo / (ms / 1e3) / 1e9 / peak,
           "p50_ms": p50, "p99_ms": p99,
           "shapes": {str(L): list(r["shape"]) for L, r in tuned.items()},
           "spread": {str(L): round(r["worst_ms"] / r["best_ms"], 3) for L, r in tuned.items() if r["best_ms"] > 0}}
    if oracle_cpu:
        out["cpu"] = oracle_batched_baseline(ws)["value"]
    return out


def served_sweep(spegg, torch, count: int = 1000, rate: float = 200.0):
    """Served parameter sweep: a seeded Poisson stream (rate jobs/s) of `count`
    jobs (N log-uniform in [1e3, 2e6], L in {64, 256}, 100-2000 generations)
    admitted by device footprint and run by continuous batching; latency is
    arrival -> finish on the server's clock.  The same jobs are then run one at
    a time (the plain path) for the same-mix comparison."""
    ws, gens, arrivals = S.served_trace(count=count, rate=rate)
    srv = spegg.Server(gens_per_tick=16)
    jobs = srv.run_trace(ws, gens, arrivals)
    infos = [srv.job_info(int(j)) for j in jobs]
    c = srv.counters()
    srv.close()
    lat = np.array([i["t_finish"] - i["t_arrival"] for i in infos])
    work = sum(w.n * i["gen"] for w, i in zip(ws, infos))
    makespan = max(i["t_finish"] for i in infos) - min(i["t_arrival"] for i in infos)
    value = work / makespan
    # steady state: the work of the jobs finishing between the 10th and 90th
    # percentile completion times, over that window (the ramp-up and the drain
    # of the last long jobs excluded)
    fin = sorted((i["t_finish"], w.n * i["gen"]) for w, i in zip(ws, infos))
    lo, hi = len(fin) // 10, (9 * len(fin)) // 10
    steady = sum(x for _, x in fin[lo + 1:hi + 1]) / max(fin[hi][0] - fin[lo][0], 1e-9)
    # the plain path on the same mix: each job created, stepped and read alone
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for w, g in zip(ws, gens):
        p = spegg.Population.from_workload(w, stats_capacity=g, stream=stream)
        p.step(g)
        p.read_stats(1, g)
        p.close()
    plain = work / (time.perf_counter() - t0)
    return {"value": value, "steady": steady, "vs_plain": value / plain, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "jobs": count, "load": rate * (work / count) / value,
            "resident": c["peak_resident"]}


def variant_population(spegg, torch, w, gens: int = 256, bytes_per_offspring=None):
    """One variant of the consumer-resource population (N = 10^6, L = 128),
    `gens` generations after 64, L2 flushed before, CUDA events on its stream."""
    stream = torch.cuda.Stream()
    pop = spegg.Population.from_workload(w, stats_capacity=gens + 128, stream=stream)
    pop.step(64)
    pop.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        flush.fill_(7)
    ms = timed_on(stream, torch, lambda: pop.step(gens))
    peak, _ = load_peaks()
    per = bytes_per_offspring if bytes_per_offspring is not None else 12 + 24 * w.words
    pop.close()
    return {"us": ms * 1e3 / gens, "frac": w.n * per * gens / (ms / 1e3) / 1e9 / peak}


def spatial_community(spegg, torch, steps: int = 200, oracle_cpu: bool = False):
    """Three-species community on a 64 x 64 torus, 814 founders per species
    and patch (1.0e7 individuals), L = 256, age classes 0/1/2, dispersal 0.05,
    200 steps; throughput in individual-steps per second."""
    c = S.spatial_community()
    stream = torch.cuda.Stream()
    g = spegg.Space(c, stream=stream, stats_capacity=steps + 8)
    g.step(3)
    g.synchronize()
    ms = timed_on(stream, torch, lambda: g.step(steps))
    st = g.read_stats(4, steps)
    ind = int(st["n_before"].sum())
    births = int(st["births"].sum())
    words = c.n_loci // 32
    # algorithmic bytes: every member's record (8W B) and age read once and
    # written once at its new place; every newborn reads two parent records
    # and is written once with its age
    algo = ind * (16 * words + 2) + births * (24 * words + 1)
    peak, _ = load_peaks()
    out = {"value": ind / (ms / 1e3), "ms": ms / steps, "frac": algo / (ms / 1e3) / 1e9 / peak}
    if oracle_cpu:
        out["cpu"] = oracle_spatial_baseline()["value"]
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
    return {"value": ind / busy * cores, "cores": cores}


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
    return {"value": ind / dt}


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
            "sample": f"first {gens} generations of the headline population, 1 thread, {dt:.1f} s"}


def r3(x):
    """Three significant digits (the bench line is kept short)."""
    if isinstance(x, float):
        return float(f"{x:.3g}")
    if isinstance(x, dict):
        return {k: r3(v) for k, v in x.items()}
    if isinstance(x, list):
        return [r3(v) for v in x]
    return x


SECTIONS = ("single", "batched", "served", "spatial", "linked", "weighted", "dominance", "continuous")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="omit the CPU oracle baselines")
    for name in SECTIONS:
        ap.add_argument(f"--no-{name}", action="store_true", help=f"omit the {name} measurement")
    ap.add_argument("--shape", default="", metavar="B,I,P",
                    help="launch shape of the headline population: threads per block, offspring per thread, lanes "
                         "per offspring; results do not depend on it")
    ap.add_argument("--only-batched", type=int, default=0, metavar="R",
                    help="run only the batched-replicates measurement on the first R replicates (profiling)")
    ap.add_argument("--served-jobs", type=int, default=1000, help="jobs of the served trace")
    ap.add_argument("--generations", type=int, default=GENERATIONS,
                    help="generations per step of the headline population (short runs for profiling)")
    args = ap.parse_args()
    set_generations(args.generations)
    workload = S.consumer_resource()
    if args.impl == "reference":
        reference_arm(args, workload)
        return
    if args.only_batched:
        import torch
        from paper_1603_09255_gb300 import build as pkg_build
        pkg_build.build()
        from paper_1603_09255_gb300 import spegg
        print(json.dumps(batched_replicates(spegg, torch, gens=args.steps, count=args.only_batched)))
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
    total_ms = max_over_ranks(sum(step_ms), device="cuda")
    st = pop.state()
    assert st["status"] == 0, f"population status {st['status']}"
    value = workload.n * GENERATIONS * args.steps * ws / (total_ms / 1000.0)

    # roofline of one generation (offspring + compaction launches, timed together)
    launches = GENERATIONS * args.steps
    avg_gen_s = total_ms / 1000.0 / launches
    peak, peak_kind = load_peaks()
    achieved = algorithmic_bytes(workload.words) * workload.n / avg_gen_s / 1e9
    traffic = MEASURED_TRAFFIC.get(kernel_source_hash())
    gen_p50, gen_p99 = per_generation_ms(stream, torch, lambda: pop.step(1), repeats=50)

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
    shape = pop.launch_shape()
    pop.close()

    cpu = rank == 0 and not args.no_cpu_baseline
    extra = {}
    if not args.no_single:
        extra["single"] = single_species(spegg, torch, cpu)
    if not args.no_batched:
        extra["batched"] = batched_replicates(spegg, torch, oracle_cpu=cpu)
    if not args.no_served:
        extra["served"] = served_sweep(spegg, torch, count=args.served_jobs)
    if not args.no_spatial:
        extra["spatial"] = spatial_community(spegg, torch, oracle_cpu=cpu)
    if not args.no_linked:
        extra["linked"] = variant_population(spegg, torch, S.with_linkage(S.consumer_resource(), 4, 1.0))
    if not args.no_weighted:
        extra["weighted"] = variant_population(spegg, torch, S.with_weights(S.consumer_resource()))
    if not args.no_dominance:
        extra["dominance"] = variant_population(spegg, torch, S.with_dominance(S.consumer_resource()))
    if not args.no_continuous:
        extra["continuous"] = variant_population(
            spegg, torch, S.continuous_trait(n=1_000_000, n_loci=128, mu=1e-3, mut_sd=0.05, env_sd=0.2), gens=64,
            bytes_per_offspring=12 + 12 * 128)
    if rank != 0:
        return
    line = {
        "metric": "individual-generations/s", "value": value, "unit": "individual-generations/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": bench_config(workload, "flushed"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "shape": list(shape)},
        "e2e": {"value": e2e_value, "unit": "individual-generations/s", "h2d_bytes_per_step": len(blob),
                "d2h_bytes_per_step": int(stats.nbytes)},
        "gpu_launches": 2 * launches,
        "clocks": clocks.summary(),
        "gen_ms": {"p50": gen_p50, "p99": gen_p99},
    }
    if cpu:
        line["cpu_baseline"] = cpu_baseline(workload)
    line["gen_ms"] = r3(line["gen_ms"])
    line.update(r3(extra))
    print(json.dumps(line, separators=(",", ":")))


if __name__ == "__main__":
    main()
