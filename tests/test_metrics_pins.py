"""Pins of the oracle's coordination counts (Section 5.2, "Key Metrics":
Cross-Agent % and Interleaved %), on hand-worked solutions whose counts follow
from the definitions by inspection, and on the undefined cases."""
import numpy as np

import oracle
import workloads


def line_instance(m, p):
    # depot at 0, customer c at 10c on a line: d(a, b) = 10 |a - b|
    n = len(p)
    coords = np.array([[10 * i, 0] for i in range(n + 1)], np.int32)
    w = workloads.Instance(coords, np.array(p, np.int32), m, 4 * m, 4)
    return oracle.OracleInstance.from_workload(w)


def sol(*routes):
    ops = np.array([o for r in routes for o in r], np.int32)
    off = np.zeros(len(routes) + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in routes])
    return ops, off


D = lambda c: 2 * c
P = lambda c: 2 * c + 1


def test_one_vehicle_adjacent_pairs_are_not_interleaved():
    I = line_instance(1, [5, 5])
    assert oracle.coordination(I, *sol([D(1), P(1), D(2), P(2)])) == (0, 0, 0)


def test_one_vehicle_nested_and_crossed_pairs():
    I = line_instance(1, [5, 5])
    assert oracle.coordination(I, *sol([D(1), D(2), P(1), P(2)]))[:2] == (0, 2)
    # D1 D2 P2 P1: customer 1 has two ops between, customer 2 none
    assert oracle.coordination(I, *sol([D(1), D(2), P(2), P(1)]))[:2] == (0, 1)


def test_cross_vehicle_interleaving_compares_next_arrival_with_pickup_completion():
    # vehicle 0: D1 (t=10) D2 (t=20); vehicle 1: P1 arrives at 10, completes at
    # max(10, 10 + p1).  Vehicle 0 reaches its next op at 20.
    ops, off = sol([D(1), D(2)], [P(1), P(2)])
    # p1 = 100: P1 completes at 110 > 20, so customer 1 is interleaved;
    # customer 2's dropoff is vehicle 0's last op, so it is not
    assert oracle.coordination(line_instance(2, [100, 100]), ops, off)[:2] == (2, 1)
    # p1 = 5: P1 completes at 15 < 20, nothing in between
    assert oracle.coordination(line_instance(2, [5, 100]), ops, off)[:2] == (2, 0)
    # p1 = 10: completes at 20, the next op is reached at 20 (not before)
    assert oracle.coordination(line_instance(2, [10, 100]), ops, off)[:2] == (2, 0)


def test_undefined_counts():
    I = line_instance(2, [5, 5])
    # precedence cycle across vehicles: P2 before D1 on vehicle 0, P1 before D2 on vehicle 1
    cr, il, st = oracle.coordination(I, *sol([P(2), D(1)], [P(1), D(2)]))
    assert st & oracle.CYCLE and cr == 2 and il == -1
    # customer 2 missing its pickup
    cr, il, st = oracle.coordination(I, *sol([D(1), P(1), D(2)], []))
    assert st & oracle.MALFORMED and (cr, il) == (-1, -1)


def test_counts_bounded_and_zero_cross_on_one_vehicle():
    w = workloads.make_instance(20, 1, 20, 20, "2x", seed=1)
    I = oracle.OracleInstance.from_workload(w)
    ops, off = workloads.precedence_candidates(20, 1, 30, seed=2)
    for k in range(30):
        cr, il, st = oracle.coordination(I, ops[k], off[k])
        assert cr == 0 and 0 <= il <= 20
    w = workloads.make_instance(20, 4, 20, 20, "5x", seed=1)
    I = oracle.OracleInstance.from_workload(w)
    ops, off = workloads.precedence_candidates(20, 4, 30, seed=3)
    for k in range(30):
        cr, il, st = oracle.coordination(I, ops[k], off[k])
        assert 0 <= cr <= 20 and 0 <= il <= 20
