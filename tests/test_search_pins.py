"""Pins of the oracle's repair operators (Section 4.2.3) that follow from the
definitions alone: regret-k sums (c_i - c_1) over the k best per-vehicle
options, so with m = 2 regret-m is regret-2, and with m = 3 regret-3 is
regret-m.  A search that enables one operator draws it every iteration, so the
paired runs must agree step for step."""
import numpy as np
import pytest

import oracle
import workloads


def run(w, iters, seed, mask):
    I = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(I, w.coords)
    return oracle.alns_run(I, init[0], init[1], oracle.alns_params(iters, 4, 4, mask), seed)


def same(a, b):
    assert np.array_equal(a["trace"], b["trace"])
    for f in ("accepted", "improved", "new_best", "reheats", "rejected_infeasible", "z_best"):
        assert getattr(a["stats"], f) == getattr(b["stats"], f), f
    assert np.array_equal(a["best_ops"], b["best_ops"]) and np.array_equal(a["best_off"], b["best_off"])


@pytest.mark.parametrize("seed", range(3))
def test_regret_m_is_regret_2_for_two_vehicles(seed):
    w = workloads.make_instance(14, 2, 6, 4, "2x", seed=seed)
    same(run(w, 25, seed, 8), run(w, 25, seed, 2))


@pytest.mark.parametrize("seed", range(3))
def test_regret_3_is_regret_m_for_three_vehicles(seed):
    w = workloads.make_instance(15, 3, 6, 3, "5x", seed=seed + 7)
    same(run(w, 25, seed, 4), run(w, 25, seed, 8))


def test_regret_operators_differ_somewhere():
    # with more vehicles the regret definitions part ways on some instance
    diffs = 0
    for seed in range(6):
        w = workloads.make_instance(16, 5, 8, 3, "2x", seed=seed)
        a, b = run(w, 15, seed, 2), run(w, 15, seed, 8)
        diffs += int(not np.array_equal(a["trace"], b["trace"]))
    assert diffs > 0
