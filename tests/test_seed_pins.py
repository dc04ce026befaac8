"""Pins of the construction seeds of the BRKGA warm start (Section 4.4.4):
nearest neighbour, load-balanced and shortest processing time, each a
chromosome whose drops all come before its pickups in one customer order.
Checked against what the definitions fix: the priorities are a permutation
with each pickup n places after its drop; with one ample vehicle the decoder
(pinned elsewhere) gives exactly that order, all drops then all pickups; the
orders are sorted by p (SPT) and by workload 2 d(0,c) + p_c (load-balanced);
the nearest-neighbour order is a nearest-neighbour tour of the distance matrix;
the load-balanced hints follow a least-loaded assignment."""
import numpy as np
import pytest

import oracle
import workloads


def order_of(keys, n):
    pr = keys[: 2 * n]
    drops = np.argsort(pr[0::2], kind="stable") + 1
    return [int(c) for c in drops]


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("h", [0, 1, 2])
def test_priorities_are_drops_then_pickups(h, layout):
    n, m = 17, 3
    w = workloads.make_instance(n, m, 20, 5, "1R10", seed=h)
    I = oracle.OracleInstance.from_workload(w)
    keys = oracle.seed_chromosome(I, h, layout)
    assert keys.shape[0] == oracle.key_length(I, layout)
    r = np.rint(keys[: 2 * n].astype(np.float64) * 2 * n).astype(int)
    assert sorted(r[0::2]) == list(range(n)) and np.array_equal(r[1::2], r[0::2] + n)
    assert (keys >= 0).all() and (keys < 1).all()


@pytest.mark.parametrize("h", [0, 1, 2])
def test_one_vehicle_decode_is_the_order(h):
    n = 12
    w = workloads.make_instance(n, 1, n, n, "2x", seed=5)
    I = oracle.OracleInstance.from_workload(w)
    keys = oracle.seed_chromosome(I, h, 0)
    order = order_of(keys, n)
    ops, off, z, un, fit = oracle.decode(I, keys, 0)
    assert un == 0
    assert list(ops) == [2 * c for c in order] + [2 * c + 1 for c in order]


def test_orders_follow_their_rules():
    n, m = 40, 4
    w = workloads.make_instance(n, m, 40, 8, "1R20", "clustered", seed=3)
    I = oracle.OracleInstance.from_workload(w)
    d = oracle.euc2d(w.coords).astype(np.int64)
    p = w.p.astype(np.int64)
    spt = order_of(oracle.seed_chromosome(I, 2, 0), n)
    assert all((p[a - 1], a) < (p[b - 1], b) for a, b in zip(spt, spt[1:]))
    lb = order_of(oracle.seed_chromosome(I, 1, 0), n)
    wl = {c: 2 * d[0, c] + p[c - 1] for c in range(1, n + 1)}
    assert all((-wl[a], a) < (-wl[b], b) for a, b in zip(lb, lb[1:]))
    nn = order_of(oracle.seed_chromosome(I, 0, 0), n)
    prev, left = 0, set(range(1, n + 1))
    for c in nn:
        assert (d[prev, c], c) == min((d[prev, x], x) for x in left)
        left.remove(c)
        prev = c


def test_load_balanced_hints_are_least_loaded():
    n, m = 30, 5
    w = workloads.make_instance(n, m, 30, 6, "5x", seed=9)
    I = oracle.OracleInstance.from_workload(w)
    d = oracle.euc2d(w.coords).astype(np.int64)
    keys = oracle.seed_chromosome(I, 1, 1)
    hints = keys[2 * n:].astype(np.float64)
    veh = np.minimum(np.floor(hints * m), m - 1).astype(int)
    assert np.array_equal(veh[0::2], veh[1::2])
    load = [0] * m
    for c in order_of(keys, n):
        v = veh[2 * (c - 1)]
        assert load[v] == min(load) and v == load.index(min(load))
        load[v] += 2 * d[0, c] + w.p[c - 1]
    # nearest neighbour and SPT hint vehicle 0 everywhere
    for h in (0, 2):
        k = oracle.seed_chromosome(I, h, 1)
        assert (np.floor(k[2 * n:].astype(np.float64) * m) == 0).all()
