"""Pins of the oracle's multi-instance ALNS (Section 4.2.1: independent
replicas with a best-of-all import every sync_every iterations), checked
against the single-instance oracle run (pinned elsewhere) and the import's
definition."""
import numpy as np
import pytest

import oracle
import workloads


def setup(n=24, m=3, seed=2):
    w = workloads.make_instance(n, m, 8, 4, "5x", seed=seed)
    oi = oracle.OracleInstance.from_workload(w)
    return oi, oracle.initial_solution(oi, w.coords)


def test_one_replica_is_the_single_run():
    oi, init = setup()
    P = oracle.alns_params(40, 3, 6, 15, destroy_mask=63, ls_pickup_every=7, ls_relocate_every=11)
    one = oracle.alns_run(oi, init[0], init[1], P, 9)
    rep = oracle.alns_run_replicas(oi, init[0], init[1], P, 9, 1, 10)
    assert np.array_equal(rep["traces"][0], one["trace"]) and rep["imports"] == 0
    assert np.array_equal(rep["best_ops"], one["best_ops"]) and rep["stats"][0].z_best == one["stats"].z_best


def test_replicas_without_a_checkpoint_are_independent():
    oi, init = setup(30, 4, 3)
    P = oracle.alns_params(30)
    rep = oracle.alns_run_replicas(oi, init[0], init[1], P, 4, 4, 1000)
    one = oracle.alns_run(oi, init[0], init[1], P, 4)
    assert np.array_equal(rep["traces"][0], one["trace"]) and rep["imports"] == 0
    zb = [st.z_best for st in rep["stats"]]
    assert rep["best_replica"] == int(np.argmin(zb))
    assert oracle.evaluate(oi, rep["best_ops"], rep["best_off"]) == (min(zb), 0)
    # different streams give different searches
    assert len({tuple(t) for t in rep["traces"]}) > 1


@pytest.mark.parametrize("sync", [5, 8])
def test_checkpoints_import_the_best_of_all(sync):
    oi, init = setup(24, 3, 5)
    R, iters = 4, 24
    P = oracle.alns_params(iters, 3, 6, 15, destroy_mask=63, ls_pickup_every=0, ls_relocate_every=0)
    rep = oracle.alns_run_replicas(oi, init[0], init[1], P, 7, R, sync)
    # replay the checkpoints from the traces (a replica's best is the least
    # makespan it has held): at each, every replica behind the best of all is
    # one import, and all continue from that best
    best_so_far = np.minimum.accumulate(rep["traces"], axis=1)
    imports = 0
    z_best_at = np.full(R, rep["stats"][0].z_init)
    for it in range(1, iters + 1):
        z_best_at = np.minimum(z_best_at, rep["traces"][:, it - 1])
        if it % sync == 0:
            g = int(np.min(z_best_at))
            imports += int((z_best_at > g).sum())
            z_best_at[:] = g
    assert rep["imports"] == imports
    assert min(st.z_best for st in rep["stats"]) == int(best_so_far.min())
