"""The evaluator's semantics against the paper's MILP (Section 3.1, Eqs. 1-22).

The MILP is written out constraint by constraint and solved with HiGHS for
tiny instances; its optimum must equal the best makespan over every candidate
the evaluator scores feasible, restricted to what the MILP can express: each
vehicle visits a customer at most once (a vehicle doing both operations does
them in one visit, drop then pickup), every vehicle leaves the depot (Eq. 2),
every vehicle starts full (Eq. 13) with a pool large enough not to bind, and a
visit that both drops and picks up needs room for the pickup before it drops
(Eq. 18).  Eq. 12 is applied to arcs into customers; the return arc is Eq. 21.
"""
import itertools

import numpy as np
import pytest

import oracle

opt = pytest.importorskip("scipy.optimize")


def solve_milp(d, p, m, k):
    n = len(p)
    C = list(range(1, n + 1))
    N = [0] + C
    V = list(range(m))
    M = 10 * (int(d.sum()) + int(sum(p)) + 1)
    idx = {}

    def var(name):
        if name not in idx:
            idx[name] = len(idx)
        return idx[name]

    for v in V:
        for i in N:
            for j in N:
                var(("x", i, j, v))
        for c in C:
            var(("y", c, v)); var(("dl", c, v)); var(("pk", c, v)); var(("u", c, v))
        for i in N:
            var(("t", i, v)); var(("td", i, v)); var(("q", i, v))
        var(("tr", v))
    for c in C:
        var(("TD", c)); var(("TP", c))
    var(("T",))
    nv = len(idx)
    rows, lo, hi = [], [], []

    def add(coefs, lb, ub):
        r = np.zeros(nv)
        for name, a in coefs:
            r[idx[name]] += a
        rows.append(r); lo.append(lb); hi.append(ub)

    inf = np.inf
    for c in C:                                                    # Eq. 1
        add([(("dl", c, v), 1) for v in V], 1, 1)
        add([(("pk", c, v), 1) for v in V], 1, 1)
        add([(("TP", c), 1), (("TD", c), -1)], p[c - 1], inf)     # Eq. 9
    for v in V:
        add([(("x", 0, j, v), 1) for j in C], 1, 1)                # Eq. 2
        add([(("x", i, 0, v), 1) for i in C], 1, 1)
        add([(("t", 0, v), 1)], 0, 0)                              # Eq. 3
        add([(("td", 0, v), 1)], 0, 0)
        add([(("q", 0, v), 1)], k, k)                              # Eq. 13
        for c in C:
            add([(("x", i, c, v), 1) for i in N] + [(("y", c, v), -1)], 0, 0)   # Eq. 4
            add([(("x", c, j, v), 1) for j in N] + [(("y", c, v), -1)], 0, 0)
            add([(("dl", c, v), 1), (("y", c, v), -1)], -inf, 0)  # Eq. 6
            add([(("pk", c, v), 1), (("y", c, v), -1)], -inf, 0)
            # Eq. 7: t - M(1-dl) <= TD <= t + M(1-dl)
            add([(("t", c, v), 1), (("dl", c, v), M), (("TD", c), -1)], -inf, M)
            add([(("TD", c), 1), (("t", c, v), -1), (("dl", c, v), M)], -inf, M)
            # Eq. 8
            add([(("td", c, v), 1), (("pk", c, v), M), (("TP", c), -1)], -inf, M)
            add([(("TP", c), 1), (("td", c, v), -1), (("pk", c, v), M)], -inf, M)
            add([(("td", c, v), 1), (("t", c, v), -1)], 0, inf)     # Eq. 10
            # Eq. 11: td >= t + p(dl + pk - 1)
            add([(("td", c, v), 1), (("t", c, v), -1), (("dl", c, v), -p[c - 1]), (("pk", c, v), -p[c - 1])],
                -p[c - 1], inf)
            # Eq. 21
            add([(("tr", v), 1), (("td", c, v), -1), (("x", c, 0, v), -M)], d[c, 0] - M, inf)
            add([(("u", c, v), 1)], 1, n)                           # Eq. 19
        for i in N:
            add([(("x", i, i, v), 1)], 0, 0)                        # Eq. 5
            add([(("q", i, v), 1)], 0, k)                           # Eq. 14
            for j in C:
                if i == j:
                    continue
                # Eq. 12 on arcs into customers
                add([(("t", j, v), 1), (("td", i, v), -1), (("x", i, j, v), -M)], d[i, j] - M, inf)
                # Eqs. 15-16
                add([(("q", j, v), 1), (("q", i, v), -1), (("dl", j, v), 1), (("pk", j, v), -1),
                     (("x", i, j, v), -M)], -M, inf)
                add([(("q", j, v), 1), (("q", i, v), -1), (("dl", j, v), 1), (("pk", j, v), -1),
                     (("x", i, j, v), M)], -inf, M)
                # Eq. 17 and Eq. 18
                add([(("q", i, v), 1), (("dl", j, v), -1), (("x", i, j, v), -M)], -M, inf)
                add([(("q", i, v), 1), (("pk", j, v), 1), (("x", i, j, v), M)], -inf, k + M)
        for i in C:
            for j in C:
                if i != j:                                          # Eq. 20
                    add([(("u", i, v), 1), (("u", j, v), -1), (("x", i, j, v), n)], -inf, n - 1)
        add([(("T",), 1), (("tr", v), -1)], 0, inf)                # Eq. 22
    integ = np.zeros(nv)
    for name, col in idx.items():
        if name[0] in ("x", "y", "dl", "pk"):
            integ[col] = 1
    lb = np.zeros(nv)
    ub = np.full(nv, np.inf)
    for name, col in idx.items():
        if name[0] in ("x", "y", "dl", "pk"):
            ub[col] = 1
    cost = np.zeros(nv)
    cost[idx[("T",)]] = 1
    res = opt.milp(cost, constraints=opt.LinearConstraint(np.array(rows), lo, hi), integrality=integ,
                   bounds=opt.Bounds(lb, ub), options={"time_limit": 60})
    if res.status == 2:                       # infeasible
        return None
    assert res.status == 0, res.message
    return res.fun


def milp_expressible(routes, k):
    for r in routes:
        if not r:
            return False                                  # Eq. 2: every vehicle leaves
        custs = [o >> 1 for o in r]
        # one visit per customer: both operations adjacent, drop first
        for i, c in enumerate(custs):
            if custs.count(c) == 2:
                j = custs.index(c, i + 1) if custs.index(c) == i else None
                if j is not None and (j != i + 1 or r[i] & 1):
                    return False
        s = k
        i = 0
        while i < len(r):
            if i + 1 < len(r) and custs[i + 1] == custs[i]:
                if s < 1 or s + 1 > k:                    # Eqs. 17-18 on a drop+pickup visit
                    return False
                i += 2
                continue
            if r[i] & 1:
                if s + 1 > k:
                    return False
                s += 1
            else:
                if s < 1:
                    return False
                s -= 1
            i += 1
    return True


def bruteforce_milp_space(I, k):
    n, m = I.n, I.m
    best = None
    ops_all = list(range(2, 2 * n + 2))
    for perm in itertools.permutations(ops_all):
        for cuts in itertools.combinations(range(1, 2 * n), m - 1):
            bounds = (0,) + cuts + (2 * n,)
            routes = [list(perm[bounds[v]:bounds[v + 1]]) for v in range(m)]
            if not milp_expressible(routes, k):
                continue
            z, st = oracle.evaluate(I, np.array(perm, np.int32), np.array(bounds, np.int32))
            if st & (oracle.CYCLE | oracle.MALFORMED):
                continue
            best = z if best is None or z < best else best
    return best


@pytest.mark.parametrize("seed,n,m,k", [(0, 2, 2, 2), (1, 3, 2, 2), (2, 3, 2, 3), (4, 2, 2, 1), (5, 3, 2, 2),
                                        (6, 3, 2, 3), (3, 3, 1, 2)])
def test_evaluator_optimum_equals_milp(seed, n, m, k):
    # with m = 1 both sides must be infeasible: a full vehicle's first visit can
    # only drop, and without revisits no one can collect that resource
    rng = np.random.default_rng(seed)
    coords = rng.integers(0, 25, size=(n + 1, 2)).astype(np.int32)
    p = rng.integers(0, 30, size=n).astype(np.int32)
    d = oracle.euc2d(coords)
    I = oracle.OracleInstance(d, p, m, R=m * k, Q=k, load_full=True)
    bf = bruteforce_milp_space(I, k)
    z = solve_milp(d.astype(np.int64), [int(x) for x in p], m, k)
    assert (bf is None) == (z is None), (bf, z)
    if bf is not None:
        assert abs(z - bf) < 1e-6, (z, bf)
