"""Pins of the oracle's search loops against what their definitions fix,
with fitness recomputed by the pinned decoder:
  * BRKGA (Section 4.4.3): the population after one generation starts with
    the previous one's N_e best chromosomes, copied exactly (fitness, then
    index); every crossover gene is the same gene of some previous
    chromosome; mutants are fresh keys in [0, 1);
  * ALNS (Algorithm 1, Section 4.2.4): with no reheat, the temperature after
    k iterations is T0 z_init alpha^k up to rounding, and a search that
    accepts nothing keeps its start as current and best."""
import math

import numpy as np
import pytest

import oracle
import workloads


@pytest.mark.parametrize("layout", [0, 1])
def test_brkga_one_generation(layout):
    w = workloads.make_instance(15, 3, 6, 4, "2x", seed=2)
    I = oracle.OracleInstance.from_workload(w)
    pop, elite, mutant = 40, 0.2, 0.1
    P1 = oracle.brkga_params(pop, 1, elite, mutant, layout=layout)
    P2 = oracle.brkga_params(pop, 2, elite, mutant, layout=layout)
    warm = oracle.initial_solution(I, w.coords)
    g0 = oracle.brkga_run(I, P1, warm[0], warm[1], 5)["keys"]          # the initial population
    g1 = oracle.brkga_run(I, P2, warm[0], warm[1], 5)["keys"]          # after one generation
    fit = [oracle.decode(I, g0[s], layout)[4] for s in range(pop)]
    order = sorted(range(pop), key=lambda s: (fit[s], s))
    ne, nm = int(math.floor(elite * pop)), int(math.floor(mutant * pop))
    for k in range(ne):
        assert np.array_equal(g1[k].view(np.uint32), g0[order[k]].view(np.uint32))
    for s in range(ne, pop - nm):
        for gi in range(g1.shape[1]):
            assert g1[s, gi] in g0[:, gi]
    assert (g1[pop - nm:] >= 0).all() and (g1[pop - nm:] < 1).all()
    # the trace is the best fitness of each generation
    tr = oracle.brkga_run(I, P2, warm[0], warm[1], 5)["trace"]
    assert tr[0] == fit[order[0]] and tr[1] <= tr[0]


def test_alns_temperature_schedule():
    w = workloads.make_instance(20, 3, 8, 4, "5x", seed=3)
    I = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(I, w.coords)
    iters = 150
    o = oracle.alns_run(I, init[0], init[1], oracle.alns_params(iters, ls_pickup_every=0, ls_relocate_every=0), 1)
    st = o["stats"]
    assert st.reheats == 0
    expect = 0.30 * st.z_init * 0.9998 ** iters
    assert abs(st.T_final - expect) <= 1e-9 * expect


def test_alns_without_acceptance_keeps_its_start():
    # T0 = 0 accepts no worsening move; on a one-customer instance every
    # repair rebuilds the only (optimal) schedule, so nothing improves either
    w = workloads.make_instance(1, 1, 1, 1, "base", seed=4)
    I = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(I, w.coords)
    P = oracle.alns_params(20, ls_pickup_every=0, ls_relocate_every=0)
    P.T0 = 0.0
    o = oracle.alns_run(I, init[0], init[1], P, 2)
    z0 = oracle.evaluate(I, *init)[0]
    assert o["stats"].z_best == z0 and o["stats"].improved == 0
    assert np.array_equal(o["best_ops"], init[0]) and (o["trace"] == z0).all()


def _generation_pair(rho, layout=0, pop=48, seed=6):
    w = workloads.make_instance(12, 3, 6, 4, "2x", seed=7)
    I = oracle.OracleInstance.from_workload(w)
    warm = oracle.initial_solution(I, w.coords)
    P1 = oracle.brkga_params(pop, 1, 0.25, 0.125, rho=rho, layout=layout)
    P2 = oracle.brkga_params(pop, 2, 0.25, 0.125, rho=rho, layout=layout)
    g0 = oracle.brkga_run(I, P1, warm[0], warm[1], seed)["keys"]
    g1 = oracle.brkga_run(I, P2, warm[0], warm[1], seed)["keys"]
    fit = [oracle.decode(I, g0[s], layout)[4] for s in range(pop)]
    order = sorted(range(pop), key=lambda s: (fit[s], s))
    ne, nm = int(math.floor(0.25 * pop)), int(math.floor(0.125 * pop))
    return g0, g1, order, ne, nm


def _rows(a):
    return [r.view(np.uint32).tobytes() for r in a]


@pytest.mark.parametrize("layout", [0, 1])
def test_crossover_rho_one_copies_the_elite_parent(layout):
    """Section 4.4.3: each gene comes from the elite parent with probability
    rho.  With rho = 1 every child is a copy of one of the previous N_e best
    (a draw u in [0, 1) is always below 1), and the copies do not all come
    from one parent."""
    g0, g1, order, ne, nm = _generation_pair(1.0, layout)
    pop = g0.shape[0]
    elite = set(_rows(g0[order[:ne]]))
    rest = set(_rows(g0[order[ne:]]))
    kids = _rows(g1[ne:pop - nm])
    assert all(k in elite for k in kids)
    assert not any(k in rest for k in kids)
    assert len(set(kids)) > 1


@pytest.mark.parametrize("layout", [0, 1])
def test_crossover_rho_zero_copies_the_other_parent(layout):
    """With rho = 0 no gene comes from the elite parent: every child copies one
    chromosome from outside the previous N_e best."""
    g0, g1, order, ne, nm = _generation_pair(0.0, layout)
    pop = g0.shape[0]
    elite = set(_rows(g0[order[:ne]]))
    rest = set(_rows(g0[order[ne:]]))
    kids = _rows(g1[ne:pop - nm])
    assert all(k in rest for k in kids)
    assert not any(k in elite for k in kids)
    assert len(set(kids)) > 1


def test_crossover_bias_is_rho():
    """rho = 0.7: each child is explained by one (elite, other) parent pair,
    and where the two parents differ the child takes the elite gene about 70%
    of the time (about 1000 such genes here: 0.7 +- 0.05 is beyond 3 sigma)."""
    g0, g1, order, ne, nm = _generation_pair(0.7, pop=64, seed=8)
    pop = g0.shape[0]
    E, O = g0[order[:ne]], g0[order[ne:]]
    took_e = total = 0
    for child in g1[ne:pop - nm]:
        pairs = [(e, o) for e in range(ne) for o in range(len(O))
                 if np.all((child == E[e]) | (child == O[o]))]
        assert pairs, "a child not made from an (elite, other) pair"
        e, o = pairs[0]
        diff = E[e] != O[o]
        took_e += int(np.sum(child[diff] == E[e][diff]))
        total += int(np.sum(diff))
    assert total > 800
    assert abs(took_e / total - 0.7) < 0.05, took_e / total
