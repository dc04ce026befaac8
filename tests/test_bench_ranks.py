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
