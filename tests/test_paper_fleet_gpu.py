"""GPU parity on instances built by the paper's own rules (Section 5.1: its
fleets m = 3, Q = 5 below 24 customers and m = 6, Q = 4 from 24 on; its
processing-time variants; every vehicle leaving full, LOAD_FULL): evaluation,
ALNS and BRKGA trajectories and the coordination counts, against the oracle."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pair(vrp, w):
    return vrp.Instance.from_workload(w, load_full=True), oracle.OracleInstance.from_workload(w, load_full=True)


@pytest.mark.parametrize("n,variant", [(20, "base"), (23, "1R10"), (24, "5x"), (150, "1R20")])
def test_evaluate_and_coordination(vrp, n, variant):
    w = workloads.make_paper_instance(n, variant, "clustered" if n > 100 else "uniform", seed=n)
    inst, oi = pair(vrp, w)
    ops, off = workloads.precedence_candidates(n, w.m, 513, seed=n)
    z, st = vrp.evaluate(inst, dev(ops), dev(off))
    vrp.sync(inst)
    zo, so = oracle.evaluate_batch(oi, ops, off)
    assert np.array_equal(z.cpu().numpy(), zo) and np.array_equal(st.cpu().numpy().astype(np.uint32), so)
    cr, il = vrp.coordination(inst, dev(ops), dev(off))
    cr, il = cr.cpu().numpy(), il.cpu().numpy()
    for k in range(0, 513, 16):
        assert (cr[k], il[k]) == oracle.coordination(oi, ops[k], off[k])[:2]


@pytest.mark.parametrize("n,variant", [(20, "5x"), (30, "1R20")])
def test_alns_trajectory(vrp, n, variant):
    w = workloads.make_paper_instance(n, variant, seed=3)
    inst, oi = pair(vrp, w)
    init = oracle.initial_solution(oi, w.coords)
    g = vrp.alns_run(inst, vrp.alns_params(40, 3, 6, 15, destroy_mask=63), seed=2, init=init)
    o = oracle.alns_run(oi, init[0], init[1], oracle.alns_params(40, 3, 6, 15, destroy_mask=63), 2)
    assert np.array_equal(g["trace"], o["trace"])
    assert g["stats"].z_best == o["stats"].z_best
    assert np.array_equal(g["best_ops"], o["best_ops"]) and np.array_equal(g["best_off"], o["best_off"])
    assert oracle.evaluate(oi, g["best_ops"], g["best_off"]) == (g["z_best"], 0)


@pytest.mark.parametrize("layout", [0, 1])
def test_brkga_trajectory(vrp, layout):
    w = workloads.make_paper_instance(24, "2x", seed=5)
    inst, oi = pair(vrp, w)
    wo, wf = oracle.initial_solution(oi, w.coords)
    g = vrp.brkga_run(inst, vrp.brkga_params(64, 12, layout=layout), seed=1, warm=(wo, wf), final_keys=True)
    o = oracle.brkga_run(oi, oracle.brkga_params(64, 12, layout=layout), wo, wf, 1)
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["keys"].cpu().numpy().view(np.uint32), o["keys"].view(np.uint32))
    assert oracle.evaluate(oi, g["best_ops"], g["best_off"]) == (g["z_best"], 0)
