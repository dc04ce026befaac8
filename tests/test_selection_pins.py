"""Pins of the oracle's repair selection (Section 4.2.3) against a brute force
written here from the definitions, on small partial solutions:

  * the insertion of customer c at drop gap (a, i) and pickup gap (b, j) is
    built here (gaps numbered route by route, gap i of route v before its
    i-th op, flat index row * G + col with G = ops + m);
  * each insertion is scored with the pinned evaluator: it is feasible when
    the evaluator gives no status bit (the partial solutions here are
    feasible, so that is the oracle's rule of judging the two receiving
    routes and the pool), Delta z is the makespan change, Delta travel the
    change of total route length computed here leg by leg;
  * greedy inserts the least (Delta z, Delta travel, flat index), ties
    between customers to the smaller id;
  * regret-k takes, per customer, the best insertion whose drop goes to each
    vehicle (2^40 where a vehicle has none), sorts those Delta z values and
    sums c_i - c_1 over the k best (options past m count 2^40); the largest
    regret wins, ties to the smaller id, and the customer goes to its own
    best insertion (k = 2, 3 or m).

Each step of a whole repair is compared: the oracle run for s steps must
equal s brute-force steps.
"""
import numpy as np
import pytest

import oracle
import workloads

INF = 1 << 40


def gaps(off):
    out = []
    for v in range(len(off) - 1):
        for i in range(off[v + 1] - off[v] + 1):
            out.append((v, i))
    return out


def insert(ops, off, c, a, i, b, j):
    routes = [list(ops[off[v]:off[v + 1]]) for v in range(len(off) - 1)]
    ra = routes[a]
    if a == b:
        # pickup gap j counts positions of the route before the drop went in
        r = ra[:i] + [2 * c] + ra[i:]
        jj = j + (1 if j >= i else 0)
        r = r[:jj] + [2 * c + 1] + r[jj:]
        routes[a] = r
    else:
        routes[a] = ra[:i] + [2 * c] + ra[i:]
        rb = routes[b]
        routes[b] = rb[:j] + [2 * c + 1] + rb[j:]
    nops = [o for r in routes for o in r]
    noff = np.cumsum([0] + [len(r) for r in routes]).astype(np.int32)
    return np.array(nops, np.int32), noff


def travel(d, ops, off):
    t = 0
    for v in range(len(off) - 1):
        r = ops[off[v]:off[v + 1]]
        if len(r) == 0:
            continue
        loc = 0
        for o in r:
            t += int(d[loc, o >> 1])
            loc = o >> 1
        t += int(d[loc, 0])
    return t


def options(I, ops, off, c):
    """Every feasible insertion of c: (dz, dt, flat, drop vehicle, ops', off')."""
    z0, st0 = oracle.evaluate(I, ops, off, allow_partial=True)
    assert st0 == 0
    t0 = travel(I.d, ops, off)
    gl = gaps(off)
    G = len(gl)
    out = []
    for row, (a, i) in enumerate(gl):
        for col, (b, j) in enumerate(gl):
            if a == b and j < i:
                continue                   # the pickup would come before its drop
            no, nf = insert(ops, off, c, a, i, b, j)
            z, st = oracle.evaluate(I, no, nf, allow_partial=True)
            if st:
                continue
            out.append((z - z0, travel(I.d, no, nf) - t0, row * G + col, a, no, nf))
    return out


def brute_step(I, ops, off, removed, rule):
    """One repair step by brute force; returns (customer, ops', off')."""
    best = None
    for c in sorted(removed):
        opts = options(I, ops, off, c)
        assert opts, "every customer has a feasible insertion in these cases"
        own = min(opts, key=lambda o: o[:3])
        if rule == "greedy":
            key = (own[0], own[1], own[2], c)
        else:
            k = {"regret2": 2, "regret3": 3, "regretm": I.m}[rule]
            per = []
            for v in range(I.m):
                mine = [o for o in opts if o[3] == v]
                per.append(min(mine, key=lambda o: o[:3])[0] if mine else INF)
            per.sort()
            regret = sum((per[i] if i < I.m else INF) - per[0] for i in range(k))
            key = (-regret, c)
        if best is None or key < best[0]:
            best = (key, c, own)
    _, c, own = best
    return c, own[4], own[5]


def partial_cases():
    """Feasible partial solutions: a feasible solution with a few customers removed."""
    cases = []
    for seed, (n, m, R, Q, full) in enumerate([(7, 3, 4, 2, False), (6, 2, 4, 2, False), (7, 3, 6, 2, True),
                                               (6, 3, 3, 1, False)]):
        w = workloads.make_instance(n, m, R, Q, "2x", seed=40 + seed)
        I = oracle.OracleInstance.from_workload(w, load_full=full)
        ops, off = oracle.initial_solution(I, w.coords)
        assert oracle.evaluate(I, ops, off)[1] == 0
        rng = np.random.default_rng(seed)
        for trial in range(8):
            rem = sorted(rng.choice(np.arange(1, n + 1), size=3, replace=False).tolist())
            keep = [o for o in ops if (o >> 1) not in rem]
            routes = [[o for o in ops[off[v]:off[v + 1]] if (o >> 1) not in rem] for v in range(m)]
            noff = np.cumsum([0] + [len(r) for r in routes]).astype(np.int32)
            nops = np.array(keep, np.int32)
            if oracle.evaluate(I, nops, noff, allow_partial=True)[1] == 0:
                cases.append((I, nops, noff, rem))
            if len([cc for cc in cases if cc[0] is I]) >= 3:
                break
    # twins: customers 2 and 5 share coordinates and processing time, so their
    # insertions tie on (Delta z, Delta travel, flat index) and only the
    # customer id decides between them
    w = workloads.make_instance(6, 2, 4, 2, "2x", seed=47)
    coords, p = w.coords.copy(), w.p.copy()
    coords[5], p[4] = coords[2], p[1]
    I = oracle.OracleInstance(oracle.euc2d(coords), p, 2, 4, 2)
    ops, off = oracle.initial_solution(I, coords)
    routes = [[o for o in ops[off[v]:off[v + 1]] if (o >> 1) not in (2, 5)] for v in range(2)]
    noff = np.cumsum([0] + [len(r) for r in routes]).astype(np.int32)
    nops = np.array([o for r in routes for o in r], np.int32)
    assert oracle.evaluate(I, nops, noff, allow_partial=True)[1] == 0
    cases.append((I, nops, noff, [2, 5]))
    return cases


CASES = partial_cases()


def test_cases_exist():
    assert len(CASES) >= 8


@pytest.mark.parametrize("rule", ["greedy", "regret2", "regret3", "regretm"])
def test_repair_steps_equal_brute_force(rule):
    checked = 0
    for I, ops, off, rem in CASES:
        cur_o, cur_f, left = ops, off, list(rem)
        for step in range(1, len(rem) + 1):
            # every remaining insertion stays feasible in these cases only while
            # the partial solution is; stop the comparison where it is not
            if oracle.evaluate(I, cur_o, cur_f, allow_partial=True)[1] != 0:
                break
            c, cur_o, cur_f = brute_step(I, cur_o, cur_f, left, rule)
            left.remove(c)
            got = oracle.repair(I, rule, ops, off, rem, max_steps=step)
            assert got is not None
            assert np.array_equal(got[1], cur_f) and np.array_equal(got[0], cur_o), (rule, rem, step)
            checked += 1
    assert checked >= 12


def test_twins_tie_to_the_smaller_id():
    """With two identical customers every rule's first insertion is customer
    2's (the smaller id), at the least (Delta z, Delta travel, flat index)."""
    I, ops, off, rem = CASES[-1]
    for rule in ("greedy", "regret2", "regret3", "regretm"):
        got = oracle.repair(I, rule, ops, off, rem, max_steps=1)
        assert 4 in got[0] and 10 not in got[0], rule
        c, eo, ef = brute_step(I, ops, off, rem, rule)
        assert c == 2 and np.array_equal(got[0], eo)


def test_greedy_and_regret_disagree_somewhere():
    """The cases separate the rules: a mix-up of greedy and regret-2 (or of
    k) would not pass unnoticed."""
    differ = {("greedy", "regret2"): 0, ("regret2", "regretm"): 0, ("regret2", "regret3"): 0}
    for I, ops, off, rem in CASES:
        res = {r: oracle.repair(I, r, ops, off, rem, max_steps=1) for r in ("greedy", "regret2", "regret3",
                                                                            "regretm")}
        for a, b in differ:
            if not np.array_equal(res[a][0], res[b][0]):
                differ[(a, b)] += 1
    assert all(v > 0 for v in differ.values()), differ
