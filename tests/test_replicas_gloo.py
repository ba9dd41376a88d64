"""The multi-process path of bench.py (replicas only: one population per
rank, replicate id = rank, no exchange; the job's time is the slowest
rank's) on CPU with two gloo ranks, each advancing its replica on the oracle."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import oracle
    import spegg_synth as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.replica_workload(S.single_species(n=300, n_loci=32, mu=1e-3, seed=5), rank)
        t0 = time.perf_counter()
        st = oracle.OraclePopulation.from_workload(w).step(6)
        ms = (time.perf_counter() - t0) * 1e3 + 10.0 * rank  # rank 1 is the slow one
        worst = bench.max_over_ranks(ms)
        sig = torch.tensor([int(st["sum_raw"].sum()), int(st["s"].sum())], dtype=torch.int64)
        sigs = [torch.zeros_like(sig) for _ in range(world)]
        dist.all_gather(sigs, sig)
        out.put((rank, ms, worst, [x.tolist() for x in sigs], w.replicate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, worst0, sigs0, rep0), (r1, ms1, worst1, sigs1, rep1) = res
    assert (rep0, rep1) == (0, 1)
    assert worst0 == worst1 == max(ms0, ms1)  # every rank sees the slowest rank's time
    assert sigs0 == sigs1 and sigs0[0] != sigs0[1]  # different replicate ids: independent runs
