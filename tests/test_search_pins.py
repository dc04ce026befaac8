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


# ---- destroy operators (Section 4.2.2): properties their definitions fix ----

def sol(seed, n=24, m=4):
    w = workloads.make_instance(n, m, 2 * m, 4, "2x", seed=seed)
    I = oracle.OracleInstance.from_workload(w)
    ops, off = oracle.initial_solution(I, w.coords)
    return w, I, ops, off


def route_customers(ops, off, v):
    return {int(o) >> 1 for o in ops[off[v]:off[v + 1]]}


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("op", ["random", "worst", "shaw", "cluster"])
def test_destroy_removes_exactly_q(op, seed):
    w, I, ops, off = sol(seed)
    for q in (1, 4, 7):
        assert oracle.destroy(I, op, ops, off, q, 4, 99 + seed, q << 16)[1:].sum() == q


@pytest.mark.parametrize("seed", range(6))
def test_cluster_takes_the_nearest(seed):
    w, I, ops, off = sol(seed)
    d = oracle.euc2d(w.coords)
    rem = oracle.destroy(I, "cluster", ops, off, 6, 4, 5 + seed, 1 << 16)
    removed = np.nonzero(rem)[0]
    # the seed is the removed customer from which the other removed ones are nearest
    ok = False
    for s in removed:
        others = [c for c in removed if c != s]
        kept = [c for c in range(1, I.n + 1) if not rem[c]]
        if max(d[s, others]) <= min(d[s, kept]):
            ok = True
    assert ok


@pytest.mark.parametrize("seed", range(6))
def test_route_removal_takes_a_whole_route(seed):
    w, I, ops, off = sol(seed)
    rem = oracle.destroy(I, "route", ops, off, 5, 6, 11 + seed, 2 << 16)
    removed = set(np.nonzero(rem)[0])
    assert len(removed) >= 6
    assert any(route_customers(ops, off, v) and route_customers(ops, off, v) <= removed for v in range(I.m))


@pytest.mark.parametrize("seed", range(6))
def test_critical_path_removal_stays_on_the_bottleneck(seed):
    w, I, ops, off = sol(seed)
    times = oracle.evaluate(I, ops, off, with_times=True)[2]
    d = oracle.euc2d(w.coords)
    ret = [times[ops[off[v + 1] - 1]] + d[ops[off[v + 1] - 1] >> 1, 0] if off[v + 1] > off[v] else 0
           for v in range(I.m)]
    vb = int(np.argmax(ret))
    on_b = route_customers(ops, off, vb)
    q = min(3, len(on_b))
    rem = oracle.destroy(I, "critical", ops, off, q, 1, 3 + seed, 3 << 16)
    assert set(np.nonzero(rem)[0]) <= on_b and rem.sum() == q


def test_worst_removal_favours_the_largest_gain():
    hits = 0
    for seed in range(12):
        w, I, ops, off = sol(seed, n=16, m=3)
        z = oracle.evaluate(I, ops, off)[0]
        gains = {}
        for c in range(1, I.n + 1):
            keep = np.array([(o >> 1) != c for o in ops])
            o2 = ops[keep]
            off2 = np.array([int(np.sum(keep[:k])) for k in off], np.int32)
            gains[c] = z - oracle.evaluate(I, o2, off2, allow_partial=True)[0]
        top = max(sorted(gains), key=lambda c: gains[c])
        rem = oracle.destroy(I, "worst", ops, off, 2, 2, 40 + seed, 5 << 16)
        hits += int(rem[top])
    assert hits >= 11          # rank 1 carries 98% of the r^-6 weight on each draw
