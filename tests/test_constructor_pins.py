"""Pins of the oracle's three-phase initial solution (Section 4.2.5), each
property recomputed here from the definitions: the sweep order by exact
integer angle, sectors contiguous in it, the balancing loop's stopping rule,
the nearest-neighbour rule at every step of every route, at most b resources
out at once, feasibility, and a refinement that never makes it worse."""
import functools

import numpy as np
import pytest

import oracle
import workloads


def sweep_order(coords):
    x0, y0 = int(coords[0, 0]), int(coords[0, 1])

    def half(c):
        dx, dy = int(coords[c, 0]) - x0, int(coords[c, 1]) - y0
        return 1 if (dy < 0 or (dy == 0 and dx < 0)) else 0

    def cmp(a, b):
        ha, hb = half(a), half(b)
        if ha != hb:
            return ha - hb
        ax, ay = int(coords[a, 0]) - x0, int(coords[a, 1]) - y0
        bx, by = int(coords[b, 0]) - x0, int(coords[b, 1]) - y0
        cr = ax * by - ay * bx
        if cr != 0:
            return -1 if cr > 0 else 1
        return a - b

    return sorted(range(1, coords.shape[0]), key=functools.cmp_to_key(cmp))


CASES = [(16, 2, 4, 4, "base", "uniform"), (40, 4, 10, 5, "2x", "uniform"), (60, 5, 20, 4, "1R20", "clustered"),
         (33, 6, 12, 3, "5x", "clustered"), (7, 5, 3, 2, "base", "uniform")]


@pytest.mark.parametrize("n,m,R,Q,v,lay", CASES)
def test_phases(n, m, R, Q, v, lay):
    w = workloads.make_instance(n, m, R, Q, v, lay, seed=n)
    I = oracle.OracleInstance.from_workload(w)
    d = oracle.euc2d(w.coords).astype(np.int64)
    p = w.p.astype(np.int64)
    ops, off = oracle.initial_solution_paper(I, w.coords, 0)
    assert oracle.evaluate(I, ops, off)[1] == 0
    mp = min(m, R)
    b = min(Q, R // mp)
    order = sweep_order(w.coords)
    pos = {c: k for k, c in enumerate(order)}
    routes = [[int(o) for o in ops[off[v]:off[v + 1]]] for v in range(m)]
    assert all(not r for r in routes[mp:])
    sets = [sorted({o >> 1 for o in r}, key=lambda c: pos[c]) for r in routes[:mp]]
    # contiguous sectors in vehicle order covering the sweep
    flat = [c for s in sets for c in s]
    assert flat == order
    # balancing stopped for one of its reasons
    wl = [sum(2 * d[0, c] + p[c - 1] for c in s) for s in sets]
    if mp > 1 and 10 * mp * (max(wl) - min(wl)) >= sum(wl):
        h = int(np.argmax(wl))
        nb = [g for g in (h - 1, h + 1) if 0 <= g < mp]
        g = min(nb, key=lambda x: (wl[x], x))
        if sets[h]:
            c = sets[h][0] if g < h else sets[h][-1]
            assert wl[g] + 2 * d[0, c] + p[c - 1] >= wl[h]
    # every step of every route follows the nearest-neighbour rule
    for v in range(mp):
        t, loc, out, state, rdy = 0, 0, 0, {}, {}
        for o in routes[v]:
            cands = []
            for c in sets[v]:
                s = state.get(c, 0)
                if s == 2 or (s == 0 and out >= b):
                    continue
                fin = t + d[loc, c]
                if s == 1:
                    fin = max(fin, rdy[c])
                cands.append((fin, d[loc, c], s, 2 * c + s))
            fin, dl, s, oo = min(cands)
            assert o == oo
            c = o >> 1
            if o & 1:
                state[c], out = 2, out - 1
            else:
                state[c], out, rdy[c] = 1, out + 1, fin + p[c - 1]
            assert 0 <= out <= b
            t, loc = fin, c


@pytest.mark.parametrize("n,m,R,Q,v,lay", CASES[:4])
def test_refinement_never_worse(n, m, R, Q, v, lay):
    w = workloads.make_instance(n, m, R, Q, v, lay, seed=n)
    I = oracle.OracleInstance.from_workload(w)
    z0 = oracle.evaluate(I, *oracle.initial_solution_paper(I, w.coords, 0))[0]
    z1, st = oracle.evaluate(I, *oracle.initial_solution_paper(I, w.coords, 10))
    assert st == 0 and z1 <= z0


def test_without_coordinates_the_sweep_is_by_id():
    w = workloads.make_instance(20, 3, 9, 4, "2x", seed=1)
    I = oracle.OracleInstance.from_workload(w)
    ops, off = oracle.initial_solution_paper(I, None, 0)
    assert oracle.evaluate(I, ops, off)[1] == 0
    firsts = [sorted({int(o) >> 1 for o in ops[off[v]:off[v + 1]]}) for v in range(3)]
    assert [c for s in firsts for c in s] == list(range(1, 21))
