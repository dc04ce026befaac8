"""Pins of the oracle's periodic local search (Section 4.2.6), against facts
that do not come from it:
  * a hand-worked relocation on a line (makespans and travel worked out by
    hand; the tie on both goes to the smaller customer id);
  * one pass equals a brute force written here from the definitions: every
    move of every candidate rebuilt as Python lists and scored with the pinned
    evaluator, travel summed from the distance matrix, the least
    (makespan, travel, customer, flat gap index) applied only if it lowers the
    makespan;
  * invariants: the makespan never rises, the result is feasible, pickup
    repositioning leaves every vehicle's dropoff sequence as it was, and a
    relocated customer ends with both ops on one vehicle other than the
    bottleneck."""
import numpy as np
import pytest

import oracle
import workloads


def line(p, m):
    n = len(p)
    coords = np.array([[10 * i, 0] for i in range(n + 1)], np.int32)
    return oracle.OracleInstance.from_workload(workloads.Instance(coords, np.array(p, np.int32), m, 8 * m, 8))


def sol(*routes):
    ops = np.array([o for r in routes for o in r], np.int32)
    off = np.zeros(len(routes) + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in routes])
    return ops, off


def routes_of(ops, off):
    return [[int(o) for o in ops[off[v]:off[v + 1]]] for v in range(len(off) - 1)]


def test_hand_worked_relocation():
    # v0: D1 P1 D2 P2 (times 10, 110, 120, 220, back at 240); v1 empty.
    # Moving either customer to v1 gives makespan 140 and travel 60; customer 1 wins the tie.
    I = line([100, 100], 2)
    mv, z, ops, off = oracle.local_search(I, oracle.LS_RELOCATE, *sol([2, 3, 4, 5], []))
    assert (mv, z) == (1, 140)
    assert routes_of(ops, off) == [[4, 5], [2, 3]]


def brute_one_pass(I, d, ops, off, mode):
    m = len(off) - 1
    R = routes_of(ops, off)
    z0, st, times = oracle.evaluate(I, ops, off, with_times=True)
    assert st == 0
    ret = [times[r[-1]] + d[r[-1] >> 1, 0] if r else 0 for r in R]
    bott = int(np.argmax(ret))
    veh = {o: v for v, r in enumerate(R) for o in r}
    best = None
    n = I.n
    G = 2 * n - 2 + m
    for c in range(1, n + 1):
        vd, vp = veh[2 * c], veh[2 * c + 1]
        if mode == oracle.LS_PICKUP and not 20 * ret[vp] >= 19 * z0:
            continue
        if mode == oracle.LS_RELOCATE and bott not in (vd, vp):
            continue
        W = [[o for o in r if o >> 1 != c] for r in R]
        base = np.concatenate([[0], np.cumsum([len(r) for r in W])])
        if mode == oracle.LS_PICKUP:
            places = [(vd, R[vd].index(2 * c), b, j) for b in range(m) for j in range(len(W[b]) + 1)]
        else:
            places = [(v, i, v, j) for v in range(m) if v != bott
                      for i in range(len(W[v]) + 1) for j in range(i, len(W[v]) + 1)]
        for a, i, b, j in places:
            if a == b and j < i:
                continue
            X = [list(r) for r in W]
            if a == b:
                X[a] = W[a][:i] + [2 * c] + W[a][i:j] + [2 * c + 1] + W[a][j:]
            else:
                X[a].insert(i, 2 * c)
                X[b].insert(j, 2 * c + 1)
            xo, xf = sol(*X)
            zn, stn = oracle.evaluate(I, xo, xf)
            if stn:
                continue
            tr = 0
            for r in X:
                path = [0] + [o >> 1 for o in r] + [0] if r else []
                tr += sum(int(d[path[k], path[k + 1]]) for k in range(len(path) - 1))
            key = (zn, tr, c, (base[a] + a + i) * G + base[b] + b + j)
            if best is None or key < best[0]:
                best = (key, X)
    if best is None or best[0][0] >= z0:
        return 0, z0, R
    return 1, best[0][0], best[1]


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("n,m", [(5, 2), (7, 3), (9, 2)])
def test_one_pass_is_the_brute_force_best(mode, n, m):
    tried = 0
    for seed in range(30):
        w = workloads.make_instance(n, m, 3 * n, n, "5x" if seed % 2 else "base", seed=seed)
        I = oracle.OracleInstance.from_workload(w)
        d = oracle.euc2d(w.coords)
        ops, off = workloads.precedence_candidates(n, m, 1, seed=seed + 100)
        if oracle.evaluate(I, ops[0], off[0])[1]:
            continue
        tried += 1
        mv, z, go, gf = oracle.local_search(I, mode, ops[0], off[0], passes=1)
        bmv, bz, bR = brute_one_pass(I, d, ops[0], off[0], mode)
        assert (mv, z) == (bmv, bz)
        assert routes_of(go, gf) == bR
    assert tried >= 10


@pytest.mark.parametrize("mode", [1, 2])
def test_invariants(mode):
    moved = 0
    for seed in range(25):
        w = workloads.make_instance(14, 3, 40, 14, "2x", seed=seed)
        I = oracle.OracleInstance.from_workload(w)
        ops, off = workloads.precedence_candidates(14, 3, 1, seed=seed)
        z0, st = oracle.evaluate(I, ops[0], off[0])
        if st:
            continue
        mv, z, go, gf = oracle.local_search(I, mode, ops[0], off[0])
        assert z <= z0 and oracle.evaluate(I, go, gf) == (z, 0)
        assert (mv > 0) == (z < z0)
        moved += mv
        if mode == oracle.LS_PICKUP:
            before = [[o for o in r if not o & 1] for r in routes_of(ops[0], off[0])]
            after = [[o for o in r if not o & 1] for r in routes_of(go, gf)]
            assert before == after
        elif mv:
            # one pass at a time: the relocated customer sits on one non-bottleneck vehicle
            z1, st1, times = oracle.evaluate(I, ops[0], off[0], with_times=True)
            d = oracle.euc2d(w.coords)
            R = routes_of(ops[0], off[0])
            ret = [times[r[-1]] + d[r[-1] >> 1, 0] if r else 0 for r in R]
            bott = int(np.argmax(ret))
            mv1, _, o1, f1 = oracle.local_search(I, mode, ops[0], off[0], passes=1)
            R1 = routes_of(o1, f1)
            without = lambda RR, c: [[o for o in r if o >> 1 != c] for r in RR]
            # the relocated customer: the one whose removal makes both solutions equal
            moved_c = [c for c in range(1, 15) if without(R, c) == without(R1, c)]
            placed = lambda c: {v for v, r in enumerate(R1) if 2 * c in r or 2 * c + 1 in r}
            assert any(len(placed(c)) == 1 and bott not in placed(c) for c in moved_c)
    assert moved > 0
