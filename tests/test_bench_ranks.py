"""The multi-rank path of bench.py on CPU with two gloo ranks: each rank owns
its own shard of candidates (its seed), the job's time is the slowest rank's
(a MAX all-reduce), and the reported value is the units of all ranks over
that time.  Nothing here touches a GPU."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, "cpu")
    import workloads
    ops, off = workloads.precedence_candidates(40, 4, 8, seed=rank)
    q.put((rank, slowest, ops.tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(2):
        r, slowest, shard = q.get(timeout=120)
        got[r] = (slowest, shard)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][0] == got[1][0] == 15.0          # both ranks see the slowest rank's time
    assert got[0][1] != got[1][1]                    # each rank has its own shard


def test_whole_job_rate_and_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 7.5, "cpu") == 7.5
    assert bench.whole_job_rate(1000, 4, 2.0) == 2000.0
    assert np.isclose(bench.whole_job_rate(524288 * 5, 1, 0.035), 524288 * 5 / 0.035)


def test_summary_closes_the_line_with_every_leg():
    """The JSON line ends with a short summary of every leg's headline (the
    evaluation rate and its roofline fraction, ALNS iterations/s at n=1000 and
    n=100, BRKGA generations/s, serving), so that a reader of only the line's
    end still sees the whole metric."""
    sys.path.insert(0, ROOT)
    import bench
    line = {"value": 9.0e7, "roofline": {"frac": 0.11}, "e2e": {"value": 2.5e7},
            "plain_gpu": {"value": 6.2e6}, "ops16": {"value": 1.0e8, "e2e": {"value": 4.5e7}},
            "alns_n1000": {"value": 286.0, "iterations": 200, "roofline": {"frac": 0.016}, "pruned_frac": 0.89},
            "alns_n1000_x32": {"value": 570.0}, "alns_n100": {"value": 2600.0, "iterations": 5000},
            "brkga_n200": {"value": 2800.0, "generations": 1000}, "brkga_n200_hints": {"value": 2700.0},
            "batched_multi": {"value": 6.0e8}, "serving": {"value": 50.0, "p50_ms": 50.0, "p99_ms": 75.0},
            "serving_c5": {"completed": 19, "p50_ms": 7000.0, "p99_ms": 22000.0},
            "cpu_baseline": {"value": 9.0e5}}
    s = bench.summary_of(line)
    assert s["evals_per_s_n1000"] == 9.0e7 and s["roofline_frac"] == 0.11
    assert s["alns_n1000_iters_per_s"] == 286.0 and s["alns_n1000_iterations"] == 200
    assert s["alns_n1000_pruned_frac"] == 0.89
    assert s["alns_n100_iters_per_s"] == 2600.0 and s["alns_n100_iterations"] == 5000
    assert s["brkga_n200_gens_per_s"] == 2800.0 and s["brkga_n200_generations"] == 1000
    assert s["serving_c5_completed"] == 19 and s["cpu_oracle_evals_per_s"] == 9.0e5
    # a missing leg reads None, never an error
    assert bench.summary_of({"value": 1.0})["alns_n1000_iters_per_s"] is None
