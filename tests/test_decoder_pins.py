"""Pins of the oracle's BRKGA decoder (Algorithm 2, Section 4.4.2) and of both
chromosome layouts (Section 4.4.1), against facts that do not come from the
decoder itself:
  * whatever it schedules completely is a schedule the evaluator (Eqs. 7-23,
    pinned elsewhere) gives the same makespan, with no capacity or pool fault;
  * one customer: z = 2 d(0,1) + p_1 whoever drives (closed form);
  * one vehicle with room for everything: the route is the priority order with
    each pickup whose dropoff comes later in that order moved to the second
    pass, in priority order (the passes of Algorithm 2 reduce to this);
  * the hint layout with every hint naming vehicle h decodes exactly like the
    vehicle-key layout whose keys rank the vehicles h, h+1, ... (mod m): both
    are the cyclic tie rule;
  * the warm-start hint of vehicle v maps back to v under floor(m * alpha).
"""
import numpy as np
import pytest

import oracle
import workloads


def inst_of(w, load_full=False):
    return oracle.OracleInstance.from_workload(w, load_full=load_full)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_complete_decodes_are_evaluator_schedules(layout, seed):
    w = workloads.make_instance(14, 3, 6, 3, "2x", seed=seed)
    I = inst_of(w)
    L = oracle.key_length(I, layout)
    for keys in workloads.random_keys(40, L, seed=seed + 10):
        ops, off, z, un, fit = oracle.decode(I, keys, layout)
        assert fit == z + 10**6 * un
        if un == 0:
            assert oracle.evaluate(I, ops, off) == (z, 0)


@pytest.mark.parametrize("layout", [0, 1])
def test_single_customer_closed_form(layout):
    for seed in range(5):
        w = workloads.make_instance(1, 3, 3, 1, "base", seed=seed)
        I = inst_of(w)
        d = oracle.euc2d(w.coords)
        keys = workloads.random_keys(1, oracle.key_length(I, layout), seed=seed)[0]
        ops, off, z, un, fit = oracle.decode(I, keys, layout)
        assert un == 0 and z == 2 * int(d[0, 1]) + int(w.p[0])


@pytest.mark.parametrize("layout", [0, 1])
def test_one_vehicle_route_is_priority_order_with_late_pickups_deferred(layout):
    n = 9
    w = workloads.make_instance(n, 1, n, n, "base", seed=3)
    I = inst_of(w)
    for keys in workloads.random_keys(30, oracle.key_length(I, layout), seed=4):
        order = [int(i) + 2 for i in np.argsort(keys[: 2 * n], kind="stable")]
        rank = {o: r for r, o in enumerate(order)}
        first = [o for o in order if not (o & 1) or rank[o - 1] < rank[o]]
        second = [o for o in order if (o & 1) and rank[o - 1] > rank[o]]
        ops, off, z, un, fit = oracle.decode(I, keys, layout)
        assert un == 0
        assert list(ops) == first + second


@pytest.mark.parametrize("h", [0, 1, 4])
def test_uniform_hint_equals_cyclic_vehicle_keys(h):
    m, n = 5, 12
    w = workloads.make_instance(n, m, 8, 3, "5x", seed=h + 2)
    I = inst_of(w)
    for pri in workloads.random_keys(25, 2 * n, seed=h):
        hinted = np.concatenate([pri, np.full(2 * n, np.float32((h + 0.5) / m))]).astype(np.float32)
        vkeys = np.array([((v - h) % m) / m for v in range(m)], np.float32)
        keyed = np.concatenate([pri, vkeys]).astype(np.float32)
        a = oracle.decode(I, hinted, 1)
        b = oracle.decode(I, keyed, 0)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[0][: a[1][-1]], b[0][: b[1][-1]])
        assert a[2:] == b[2:]


@pytest.mark.parametrize("m", [1, 3, 7, 20, 32])
def test_encoded_hints_name_their_vehicles(m):
    n = 3 * m
    w = workloads.make_instance(n, m, n, n, "base", seed=m)
    I = inst_of(w)
    ops, off = workloads.precedence_candidates(n, m, 1, seed=m)
    keys = oracle.encode(I, ops[0], off[0], layout=1)
    for v in range(m):
        for o in ops[0][off[0][v]:off[0][v + 1]]:
            alpha = np.float64(keys[2 * n + o - 2])
            assert int(np.floor(alpha * m)) == v
            assert keys[2 * n + o - 2] < 1.0
