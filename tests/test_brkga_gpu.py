"""GPU parity of the BRKGA path against the CPU oracle: the decoder (segmented
key sort + Algorithm 2) chromosome by chromosome, the warm-start encoding, and
whole BRKGA runs (same counter-based draws: identical per-generation best
fitness and bit-identical final populations); decoded routes re-evaluated.
Both chromosome layouts: 2n priorities + m vehicle keys, and the paper's 4n
(priorities + per-op assignment hints, Section 4.4.1)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def decode_compare(vrp, w, keys, load_full=False, layout=0):
    import torch
    inst = vrp.Instance.from_workload(w, load_full=load_full)
    oi = oracle.OracleInstance.from_workload(w, load_full=load_full)
    ops, off, z, un, fit = [t.cpu().numpy() for t in vrp.brkga_decode(inst, torch.from_numpy(keys).cuda(), layout)]
    for i in range(keys.shape[0]):
        oo, of, oz, oun, ofit = oracle.decode(oi, keys[i], layout)
        assert (z[i], un[i], fit[i]) == (oz, oun, ofit), i
        assert np.array_equal(off[i], of), i
        assert np.array_equal(ops[i][:of[-1]], oo[:of[-1]]), i
        if oun == 0:
            # invariant: the decoder's makespan is the evaluator's
            assert oracle.evaluate(oi, oo, of) == (oz, 0)


@pytest.mark.parametrize("n,m,R,Q", [(16, 2, 4, 4), (30, 3, 6, 3), (200, 6, 20, 6), (7, 5, 2, 1)])
def test_decode_random_keys(vrp, n, m, R, Q):
    w = workloads.make_instance(n, m, R, Q, "5x", "clustered" if n == 200 else "uniform", seed=n)
    keys = workloads.random_keys(256 if n < 200 else 96, 2 * n + m, seed=1)
    keys[0, : 2 * n] = 0.5                       # all priorities tie: order by op index
    keys[1, 2 * n:] = 0.25                       # all vehicle keys tie: order by vehicle index
    decode_compare(vrp, w, keys)


def test_decode_load_full(vrp):
    w = workloads.make_instance(24, 3, 18, 6, seed=4)
    decode_compare(vrp, w, workloads.random_keys(128, 51, seed=2), load_full=True)


def test_decode_encoded_alns_solution(vrp):
    w = workloads.make_instance(40, 4, 10, 5, "2x", seed=6)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops, off = vrp.initial_solution(inst)
    keys = oracle.encode(oi, ops, off)[None, :].astype(np.float32)
    decode_compare(vrp, w, keys)


def run_pair(vrp, w, pop, gens, seed, warm=True, elite=0.2, mutant=0.1, layout=0):
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    wo, wf = oracle.initial_solution(oi, w.coords) if warm else (None, None)
    g = vrp.brkga_run(inst, vrp.brkga_params(pop, gens, elite, mutant, layout=layout), seed=seed,
                      warm=(wo, wf) if warm else None, final_keys=True)
    o = oracle.brkga_run(oi, oracle.brkga_params(pop, gens, elite, mutant, layout=layout), wo, wf, seed)
    assert np.array_equal(g["trace"], o["trace"]), (g["trace"][:10], o["trace"][:10])
    gk = g["keys"].cpu().numpy()
    assert np.array_equal(gk.view(np.uint32), o["keys"].view(np.uint32))
    assert g["best_fitness"] == o["best_fitness"]
    assert np.array_equal(g["best_ops"], o["best_ops"]) and np.array_equal(g["best_off"], o["best_off"])
    assert oracle.evaluate(oi, g["best_ops"], g["best_off"]) == (g["z_best"], 0)
    assert all(np.diff(g["trace"]) <= 0)          # elites survive: best never worsens
    return g, o


def test_brkga_small_warm(vrp):
    w = workloads.make_instance(16, 2, 4, 4, "base", seed=0)
    run_pair(vrp, w, 64, 25, seed=3)


def test_brkga_small_random_start(vrp):
    w = workloads.make_instance(20, 3, 6, 3, "2x", seed=1)
    run_pair(vrp, w, 50, 10, seed=9, warm=False, elite=0.15, mutant=0.15)


def test_brkga_n200_shape_few_generations(vrp):
    # the BRKGA workload's shape: n=200 clustered, m=6, R=20, Q=6, 5x; pop 1024, 0.2/0.1/0.7
    cfg = workloads.CONFIGS["brkga_n200"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=0)
    run_pair(vrp, w, 1024, 3, seed=0)


# ---- the paper's 4n layout: per-op assignment hints ----

@pytest.mark.parametrize("n,m,R,Q", [(16, 2, 4, 4), (30, 3, 6, 3), (200, 6, 20, 6), (7, 5, 2, 1), (50, 20, 40, 3)])
def test_decode_hint_layout_random_keys(vrp, n, m, R, Q):
    w = workloads.make_instance(n, m, R, Q, "5x", "clustered" if n == 200 else "uniform", seed=n + 1)
    keys = workloads.random_keys(256 if n < 200 else 96, 4 * n, seed=2)
    keys[0, : 2 * n] = 0.5                       # all priorities tie: order by op index
    keys[1, 2 * n:] = 0.0                        # every hint names vehicle 0
    keys[2, 2 * n:] = 1.0 - 2.0 ** -24           # every hint names vehicle m-1
    decode_compare(vrp, w, keys, layout=1)


def test_decode_hint_layout_load_full(vrp):
    w = workloads.make_instance(24, 3, 18, 6, seed=5)
    decode_compare(vrp, w, workloads.random_keys(128, 96, seed=3), load_full=True, layout=1)


def test_decode_hint_layout_encoded_alns_solution(vrp):
    w = workloads.make_instance(40, 7, 10, 5, "2x", seed=6)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops, off = vrp.initial_solution(inst)
    keys = oracle.encode(oi, ops, off, layout=1)[None, :].astype(np.float32)
    decode_compare(vrp, w, keys, layout=1)


def test_brkga_hint_layout_warm(vrp):
    w = workloads.make_instance(16, 2, 4, 4, "base", seed=0)
    run_pair(vrp, w, 64, 25, seed=3, layout=1)


def test_brkga_hint_layout_n200_shape_few_generations(vrp):
    cfg = workloads.CONFIGS["brkga_n200"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=0)
    run_pair(vrp, w, 1024, 3, seed=0, layout=1)


@pytest.mark.parametrize("layout", [0, 1])
def test_warm_population_with_construction_seeds(vrp, layout):
    # one generation leaves the initial population in place: 24 warm slots
    # cycle through the 20 variants, whose last three perturb the nearest-
    # neighbour, load-balanced and SPT seeds (Section 4.4.4)
    w = workloads.make_instance(37, 4, 10, 5, "5x", "clustered", seed=2)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    wo, wf = oracle.initial_solution(oi, w.coords)
    g = vrp.brkga_run(inst, vrp.brkga_params(160, 1, layout=layout), seed=3, warm=(wo, wf), final_keys=True)
    o = oracle.brkga_run(oi, oracle.brkga_params(160, 1, layout=layout), wo, wf, 3)
    gk = g["keys"].cpu().numpy().reshape(160, -1)
    ok = o["keys"].reshape(160, -1)
    assert np.array_equal(gk.view(np.uint32), ok.view(np.uint32))
    for h in range(3):
        base = oracle.seed_chromosome(oi, h, layout)
        assert np.abs(ok[17 + h] - base).max() <= 0.03 + 1e-6
    assert np.array_equal(g["trace"], o["trace"])
