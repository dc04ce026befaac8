"""Pins of the CPU oracle's evaluator to facts outside itself (no GPU).

Each check below is fixed by the paper or by mathematics, not by re-typing the
oracle's formulas: a hand-worked schedule, the one-customer closed form,
precedence cycles, brute-force optima against the min-max VRP and the TSP
special cases of the NP-hardness reduction (Section 3.2), the shortest-path
lower bound, an existential reading of the capacity rules, exact integer
EUC_2D, and known-answer vectors of the RNG.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def inst_from(coords, p, m, R, Q, load_full=False):
    return oracle.OracleInstance(oracle.euc2d(np.array(coords, np.int32)), np.array(p, np.int32), m, R, Q,
                                 load_full)


def test_hand_worked_schedule():
    g = json.load(open(os.path.join(GOLDEN, "hand_n3.json")))
    d = oracle.euc2d(np.array(g["coords"], np.int32))
    assert d[0, 1] == 5 and d[0, 2] == 10 and d[0, 3] == 8 and d[1, 2] == 5 and d[1, 3] == 5 and d[2, 3] == 6
    for case in g["cases"]:
        I = oracle.OracleInstance(d, g["p"], case["m"], case["R"], case["Q"], case["load_full"])
        z, st, times = oracle.evaluate(I, g["ops"], g["off"], with_times=True)
        assert (z, st) == (case["z"], case["status"]), case
        for o, t in g["times_by_op"].items():
            assert times[int(o)] == t


@pytest.mark.parametrize("seed", range(6))
def test_single_customer_closed_form(seed):
    # n=1: whoever drops and picks, the pickup leaves at d01 + p1 and returns at 2*d01 + p1
    # (asymmetric d: d01 + p1 + d10)
    rng = np.random.default_rng(seed)
    d = np.array([[0, rng.integers(1, 100)], [rng.integers(1, 100), 0]], np.int32)
    p1 = int(rng.integers(0, 200))
    I = oracle.OracleInstance(d, [p1], 2, 2, 1)
    expect = int(d[0, 1] + p1 + d[1, 0])
    assert oracle.evaluate(I, [2, 3], [0, 2, 2]) == (expect, 0)         # same vehicle
    assert oracle.evaluate(I, [2, 3], [0, 1, 2])[0] == expect            # drop on 0, pick on 1
    assert oracle.evaluate(I, [3, 2], [0, 1, 2])[0] == expect            # pick listed on vehicle 0
    assert oracle.evaluate(I, [3, 2], [0, 2, 2])[1] & oracle.CYCLE       # pick before drop, one route


def test_cross_vehicle_cycle():
    coords = [[0, 0], [10, 0], [0, 10]]
    I = inst_from(coords, [5, 5], 2, 4, 2)
    # vehicle 0: P1 then D2; vehicle 1: P2 then D1 -> each pickup waits on the other's later drop
    z, st = oracle.evaluate(I, [3, 4, 5, 2], [0, 2, 4])
    assert st & oracle.CYCLE and z == 2**31 - 1
    z, st = oracle.evaluate(I, [2, 4, 3, 5], [0, 2, 4])                  # acyclic variant
    assert st == 0 and z < 2**31 - 1


def test_malformed():
    I = inst_from([[0, 0], [1, 0], [0, 1]], [1, 1], 2, 4, 2)
    assert oracle.evaluate(I, [2, 3, 4, 4], [0, 2, 4])[1] == oracle.MALFORMED   # duplicate
    assert oracle.evaluate(I, [2, 3, 4, 9], [0, 2, 4])[1] == oracle.MALFORMED   # out of range
    assert oracle.evaluate(I, [2, 3, 4, 5], [0, 3, 2])[1] == oracle.MALFORMED   # decreasing offsets
    assert oracle.evaluate(I, [2, 3, 4, 5], [1, 2, 4])[1] == oracle.MALFORMED   # off[0] != 0
    assert oracle.evaluate(I, [2, 3, 4, 5], [0, 2, 4])[1] == 0


def exact_nint_dist(coords):
    N = len(coords)
    d = np.zeros((N, N), np.int64)
    for i in range(N):
        for j in range(N):
            s = (coords[i][0] - coords[j][0]) ** 2 + (coords[i][1] - coords[j][1]) ** 2
            r = math.isqrt(s)
            d[i, j] = r + (1 if s - r * r > r else 0)      # nint: sqrt(s) is never a half-integer
    return d


def test_euc2d_exact_integer():
    rng = np.random.default_rng(3)
    coords = rng.integers(-(1 << 20), 1 << 20, size=(40, 2)).tolist() + [[0, 0], [1, 1], [2, 2], [7, 24]]
    d = oracle.euc2d(np.array(coords, np.int32))
    assert np.array_equal(d, exact_nint_dist(coords))
    # the rounding breaks the triangle inequality: (0,0),(1,1),(2,2) -> 1 + 1 < 3
    small = oracle.euc2d(np.array([[0, 0], [1, 1], [2, 2]], np.int32))
    assert small[0, 1] + small[1, 2] < small[0, 2]


def test_euc2d_rounding_boundaries():
    # legs whose squared length sits right at a rounding tie of EUC_2D:
    # s = r^2 + r (sqrt just below r + 1/2: rounds to r) and s = r^2 + r + 1
    # (just above: rounds to r + 1), for r up to about 4000, against integer
    # arithmetic alone
    g = np.arange(0, 2900, dtype=np.int64)
    dx, dy = np.meshgrid(g, g, indexing="ij")
    sq = (dx * dx + dy * dy).ravel()
    r = np.floor(np.sqrt(sq.astype(np.float64))).astype(np.int64)
    r -= (r * r > sq)
    r += ((r + 1) * (r + 1) <= sq)
    tie = (sq - r * r == r) | (sq - r * r == r + 1)
    idx = np.nonzero(tie & (r >= 2))[0]
    pick = np.random.default_rng(5).choice(idx, size=3000, replace=False)
    pts = np.stack([dx.ravel()[pick], dy.ravel()[pick]], axis=1)
    coords = np.concatenate([[[0, 0]], pts]).astype(np.int32)
    d = oracle.euc2d(coords)
    s0, r0 = sq[pick], r[pick]
    want = r0 + (s0 - r0 * r0 > r0)
    assert np.array_equal(d[0, 1:], want) and np.array_equal(d[1:, 0], want)
    assert (want == r0).sum() > 1000 and (want == r0 + 1).sum() > 1000     # both sides of the tie


def stock_feasible_existential(route_ops, Q):
    """Vehicle feasible iff SOME start load L in [0,Q] keeps stock in [0,Q] after every
    op (drop needs a resource, pickup needs room).  Returns the least such L or None."""
    for L in range(Q + 1):
        s, ok = L, True
        for o in route_ops:
            s += 1 if o & 1 else -1
            if s < 0 or s > Q:
                ok = False
                break
        if ok:
            return L
    return None


@pytest.mark.parametrize("seed", range(4))
def test_capacity_existential_reading(seed):
    n, m = 12, 3
    w = workloads.make_instance(n, m, R=6, Q=3, seed=seed)
    I = oracle.OracleInstance.from_workload(w)
    ops, off = workloads.precedence_candidates(n, m, 200, seed)
    for i in range(200):
        z, st = oracle.evaluate(I, ops[i], off[i])
        loads = [stock_feasible_existential(ops[i][off[i][v]:off[i][v + 1]], w.Q) for v in range(m)]
        veh_bad = any(L is None for L in loads)
        assert bool(st & oracle.VEH_CAP) == veh_bad
        if not veh_bad:
            assert bool(st & oracle.POOL) == (sum(loads) > w.R)
        assert not st & oracle.CYCLE


@pytest.mark.parametrize("seed", range(4))
def test_precedence_and_lower_bound_invariants(seed):
    n, m = 30, 4
    w = workloads.make_instance(n, m, R=10, Q=5, variant="5x", seed=seed)
    I = oracle.OracleInstance.from_workload(w)
    d = oracle.euc2d(w.coords)
    sp = oracle.sp_closure(d)
    lb = max(sp[0, c] + w.p[c - 1] + sp[c, 0] for c in range(1, n + 1))
    ops, off = workloads.precedence_candidates(n, m, 100, seed)
    for i in range(100):
        z, st, t = oracle.evaluate(I, ops[i], off[i], with_times=True)
        assert not st & oracle.CYCLE
        for c in range(1, n + 1):
            assert t[2 * c + 1] >= t[2 * c] + w.p[c - 1]            # Eq. 9
            assert t[2 * c] >= sp[0, c]                             # cannot arrive earlier
        assert z >= lb


def test_bruteforce_equals_minmax_vrp_when_p_zero():
    # Section 3.2: p = 0 and ample capacity reduce VRP-RPD to the min-max VRP.
    # Manhattan distances keep the triangle inequality exact.
    rng = np.random.default_rng(11)
    for trial in range(3):
        n, m = 4, 2
        pts = rng.integers(0, 30, size=(n + 1, 2))
        d = np.abs(pts[:, None, :] - pts[None, :, :]).sum(-1).astype(np.int32)
        I = oracle.OracleInstance(d, np.zeros(n, np.int32), m, R=m * n, Q=n)
        best, _, _ = oracle.bruteforce(I)
        assert best == oracle.minmax_vrp(d, n, m)


def test_bruteforce_single_vehicle_is_tsp():
    rng = np.random.default_rng(5)
    for trial in range(3):
        n = 4
        pts = rng.integers(0, 50, size=(n + 1, 2))
        d = np.abs(pts[:, None, :] - pts[None, :, :]).sum(-1).astype(np.int32)
        I = oracle.OracleInstance(d, np.zeros(n, np.int32), 1, R=n, Q=n)
        best, _, _ = oracle.bruteforce(I)
        assert best == oracle.held_karp(d, n)


def test_bruteforce_beats_every_sampled_candidate():
    w = workloads.make_instance(3, 2, R=2, Q=2, seed=7)
    I = oracle.OracleInstance.from_workload(w)
    best, bo, bf = oracle.bruteforce(I)
    assert oracle.evaluate(I, bo, bf) == (best, 0)
    ops, off = workloads.precedence_candidates(3, 2, 500, 1)
    for i in range(500):
        z, st = oracle.evaluate(I, ops[i], off[i])
        if st == 0:
            assert z >= best


def test_partial_solution_evaluation():
    w = workloads.make_instance(6, 2, R=4, Q=3, seed=2)
    I = oracle.OracleInstance.from_workload(w)
    ops, off = workloads.precedence_candidates(6, 2, 1, 3)
    keep = [o for o in ops[0] if (o >> 1) not in (2, 5)]
    # rebuild offsets after removing customers 2 and 5
    routes = [[o for o in ops[0][off[0][v]:off[0][v + 1]] if (o >> 1) not in (2, 5)] for v in range(2)]
    po = np.array(sum(routes, []), np.int32)
    pf = np.array([0, len(routes[0]), len(po)], np.int32)
    z, st = oracle.evaluate(I, po, pf, allow_partial=True)
    assert st & oracle.MALFORMED == 0
    assert oracle.evaluate(I, po, pf, allow_partial=False)[1] == oracle.MALFORMED
    assert len(keep) == len(po)


def test_rng_known_answers():
    # SplitMix64 published outputs: seed 1234567 (five draws) and seed 0 (first draw)
    assert oracle.splitmix64_stream(1234567, 5) == [6457827717110365317, 3203168211198807973,
                                                    9817491932198370423, 4593380528125082431,
                                                    16408922859458223821]
    assert oracle.splitmix64_stream(0, 1) == [0xE220A8397B1DCDAF]
    # counter form = the (counter+1)-th sequential output
    seq = oracle.splitmix64_stream(987654321, 10)
    assert [oracle.rng(987654321, k) for k in range(10)] == seq


def test_exp_accuracy():
    xs = np.concatenate([np.linspace(-700, 0, 2001), np.linspace(0, 50, 501), [-1e-300, -1e-12, -0.5]])
    for x in xs:
        e, ref = oracle.exp(float(x)), math.exp(float(x))
        assert abs(e - ref) <= 2 * math.ulp(ref), x
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-800.0) == 0.0


def test_q_range_paper_examples():
    # Section 4.2.2: n=202 -> [5,10], n=431 -> [10,21]; small n collapses to 4
    assert oracle.q_range(202) == (5, 10)
    assert oracle.q_range(431) == (10, 21)
    for n in (16, 50, 80):
        assert oracle.q_range(n) == (4, 4)
    assert oracle.q_range(1000) == (25, 50)
