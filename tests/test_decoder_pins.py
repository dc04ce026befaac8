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


# SelectVehicle (Algorithm 2, Section 4.4.2) worked by hand.  Nodes 0 (depot),
# 1, 2 with d(0,1) = 10, d(0,2) = 3, d(1,2) = 8; p = (5, 5); two vehicles,
# room for everything.  Priorities order the ops D1, D2, P1, P2 (op index
# 2(c-1) + isPickup: D1 0, P1 1, D2 2, P2 3).
#   D1: both vehicles arrive at 10: a tie, broken by the layout's rule.
#   D2: the vehicle still at the depot arrives at 3, the other at 10 + 8 = 18:
#       the least arrival wins whatever the tie rule prefers.
#   P1 (ready 15): D1's vehicle arrives at 10, the other at 3 + 8 = 11 -> D1's.
#   P2 (ready 8): D2's vehicle arrives at 3, the other at 15 + 8 = 23 -> D2's.
# Both routes are "D P"; z = max(15 + 10, 8 + 3) = 25.
def two_vehicle_instance():
    d = np.array([[0, 10, 3], [10, 0, 8], [3, 8, 0]], np.int32)
    return oracle.OracleInstance(d, np.array([5, 5], np.int32), 2, 4, 2)


PRIO = [0.1, 0.5, 0.2, 0.6]


@pytest.mark.parametrize("layout,tail,d1_vehicle", [
    (0, [0.3, 0.7], 0),                 # vehicle keys: vehicle 0 has the lower key
    (0, [0.7, 0.3], 1),                 # vehicle 1 has the lower key
    (1, [0.2, 0.9, 0.9, 0.1], 0),       # hint of D1 = 0.2 -> floor(2 * 0.2) = vehicle 0
    (1, [0.6, 0.1, 0.1, 0.9], 1),       # hint of D1 = 0.6 -> vehicle 1; the other hints name the losers
])
def test_select_vehicle_two_vehicles(layout, tail, d1_vehicle):
    I = two_vehicle_instance()
    ops, off, z, un, fit = oracle.decode(I, np.array(PRIO + tail, np.float32), layout)
    assert un == 0 and z == 25 and fit == 25
    routes = {0: [2, 3], 1: [4, 5]} if d1_vehicle == 0 else {0: [4, 5], 1: [2, 3]}
    assert list(off) == [0, 2, 4]
    assert list(ops) == routes[0] + routes[1]


def test_select_vehicle_hint_then_cyclic_order():
    """Three vehicles; d(0,1) = 10, d(0,2) = 4, d(1,2) = 20, p = (5, 5).
      D1: all three arrive at 10; hint 0.5 -> floor(1.5) = vehicle 1.
      D2: vehicles 0 and 2 arrive at 4, vehicle 1 at 30; the hint 0.4 names
          vehicle 1, not among them, so the next in cyclic order, 2, takes it
          (the lowest index would have been 0).
      P1 (ready 15): vehicles 0 and 1 arrive at 10, vehicle 2 at 24; hint 0.9
          names vehicle 2, so the cyclic order 2 -> 0 gives vehicle 0, which
          waits to 15.
      P2 (ready 9): vehicle 2 is there at 4 and waits to 9.
    Routes: (P1), (D1), (D2 P2); z = max(15 + 10, 10 + 10, 9 + 4) = 25."""
    d = np.array([[0, 10, 4], [10, 0, 20], [4, 20, 0]], np.int32)
    I = oracle.OracleInstance(d, np.array([5, 5], np.int32), 3, 4, 2)
    keys = np.array(PRIO + [0.5, 0.9, 0.4, 0.0], np.float32)
    ops, off, z, un, fit = oracle.decode(I, keys, 1)
    assert un == 0 and z == 25
    assert list(off) == [0, 1, 2, 4] and list(ops) == [3, 2, 4, 5]
    # the same instance with vehicle keys ranking 2 < 1 < 0: D1's tie goes to
    # vehicle 2; D2 then finds 0 and 1 at 4 and takes 1 (lower key than 0);
    # P1 (ready 15): 0 arrives at 10, 1 at 4 + 20 = 24, 2 at 10 -> tie 0/2 -> 2;
    # P2 (ready 9): 0 at 4, 1 at 4, 2 at 15 + 20 = 35 -> tie 0/1 -> 1 (waits to 9)
    vk = np.array(PRIO + [0.9, 0.5, 0.1], np.float32)
    ops, off, z, un, fit = oracle.decode(I, vk, 0)
    assert un == 0 and list(off) == [0, 0, 2, 4] and list(ops) == [4, 5, 2, 3]
    assert z == max(9 + 4, 15 + 10)
