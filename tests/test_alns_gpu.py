"""GPU parity of the ALNS path against the CPU oracle: the insertion-delta
matrix element by element (oracle: full re-simulation of every entry), the
start solution, and whole ALNS trajectories (same counter-based draws, so the
per-iteration makespans, the accept/improve counts, temperature and weights
must agree exactly); every returned solution is re-evaluated by the oracle."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

INT32_MAX = 2**31 - 1


def destroyed(ops, off, m, remove):
    rem = set(int(c) for c in remove)
    routes = [[int(o) for o in ops[off[v]:off[v + 1]] if (int(o) >> 1) not in rem] for v in range(m)]
    po = np.array(sum(routes, []), np.int32)
    pf = np.zeros(m + 1, np.int32)
    pf[1:] = np.cumsum([len(r) for r in routes])
    return po, pf


def matrix_case(vrp, w, seed, n_remove, load_full=False, start="initial"):
    inst = vrp.Instance.from_workload(w, load_full=load_full)
    oi = oracle.OracleInstance.from_workload(w, load_full=load_full)
    rng = np.random.default_rng(seed)
    if start == "initial":                      # feasible start: the library constructor
        ops, off = vrp.initial_solution(inst)
    else:                                       # random acyclic routes, capacity unchecked
        ops, off = workloads.precedence_candidates(w.n, w.m, 1, seed)
        ops, off = ops[0], off[0]
    remove = rng.choice(np.arange(1, w.n + 1), size=n_remove, replace=False)
    po, pf = destroyed(ops, off, w.m, remove)
    if oracle.evaluate(oi, po, pf, allow_partial=True)[1] & oracle.CYCLE:
        pytest.skip("partial solution cyclic")
    for c in remove[:2]:
        dg, tg = vrp.insertion_matrix(inst, po, pf, int(c))
        do, to, so = oracle.insertion_matrix(oi, po, pf, int(c))
        bad = np.argwhere(dg != do)
        assert bad.size == 0, (bad[:5], dg[tuple(bad[0])], do[tuple(bad[0])], so[tuple(bad[0])])
        feas = do != INT32_MAX
        assert np.array_equal(tg[feas], to[feas])
        if start == "initial":
            assert feas.any()


@pytest.mark.parametrize("seed", range(4))
def test_matrix_c1(vrp, seed):
    cfg = workloads.CONFIGS["tiny_n16"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], seed=seed)
    matrix_case(vrp, w, seed, 4)


@pytest.mark.parametrize("seed", range(3))
def test_matrix_medium(vrp, seed):
    w = workloads.make_instance(40, 4, R=10, Q=5, variant="2x", seed=10 + seed)
    matrix_case(vrp, w, seed, 6)


@pytest.mark.parametrize("seed", range(3))
def test_matrix_random_routes(vrp, seed):
    w = workloads.make_instance(30, 3, R=40, Q=30, variant="5x", seed=20 + seed)
    matrix_case(vrp, w, seed, 5, start="random")


def test_matrix_load_full(vrp):
    w = workloads.make_instance(20, 3, R=30, Q=6, seed=5)
    matrix_case(vrp, w, 5, 5, load_full=True)


def test_matrix_shortcut_gaps(vrp):
    # nearly collinear points make nint(|xc|) + nint(|cy|) < nint(|xy|): entries on such
    # gaps go through the full re-simulation path and must still match
    coords = np.array([[0, 0], [1, 1], [2, 2], [3, 3], [4, 4], [10, 0], [0, 10], [5, 5], [7, 7]], np.int32)
    p = np.array([3, 1, 4, 1, 5, 9, 2, 6], np.int32)
    w = workloads.Instance(coords, p, 2, 4, 3)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops = np.array([2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17], np.int32)
    off = np.array([0, 8, 16], np.int32)
    for c in (2, 3, 8):
        po, pf = destroyed(ops, off, 2, [c])
        dg, tg = vrp.insertion_matrix(inst, po, pf, c)
        do, to, so = oracle.insertion_matrix(oi, po, pf, c)
        assert np.array_equal(dg, do)
        feas = do != INT32_MAX
        assert np.array_equal(tg[feas], to[feas])


def test_initial_solution_matches_oracle(vrp):
    for (n, m, R, Q) in [(16, 2, 4, 4), (100, 4, 10, 5), (200, 6, 20, 6), (1000, 20, 100, 10), (7, 5, 3, 2)]:
        w = workloads.make_instance(n, m, R, Q, "2x", "clustered" if n == 200 else "uniform", seed=n)
        inst = vrp.Instance.from_workload(w)
        oi = oracle.OracleInstance.from_workload(w)
        go, gf = vrp.initial_solution(inst)
        oo, of = oracle.initial_solution(oi, w.coords)
        assert np.array_equal(go, oo) and np.array_equal(gf, of)
        assert oracle.evaluate(oi, go, gf)[1] == 0


def run_both(vrp, w, iters, seed, q=(0, 0), mask=3, team_blocks=0, dmask=1, ls=(200, 500), load_full=False):
    inst = vrp.Instance.from_workload(w, load_full=load_full)
    oi = oracle.OracleInstance.from_workload(w, load_full=load_full)
    init = oracle.initial_solution(oi, w.coords)
    g = vrp.alns_run(inst, vrp.alns_params(iters, q[0], q[1], mask, team_blocks, destroy_mask=dmask,
                                           ls_pickup_every=ls[0], ls_relocate_every=ls[1]),
                     seed=seed, init=init)
    o = oracle.alns_run(oi, init[0], init[1], oracle.alns_params(iters, q[0], q[1], mask, destroy_mask=dmask,
                                                                 ls_pickup_every=ls[0],
                                                                 ls_relocate_every=ls[1]), seed)
    return inst, oi, g, o


def assert_same_run(oi, g, o):
    assert np.array_equal(g["trace"], o["trace"]), np.nonzero(g["trace"] != o["trace"])[0][:5]
    gs, os_ = g["stats"], o["stats"]
    for f in ("accepted", "improved", "new_best", "reheats", "rejected_infeasible", "ls_moves", "ls_new_best"):
        assert getattr(gs, f) == getattr(os_, f), f
    assert gs.z_best == os_.z_best and g["z_best"] == os_.z_best
    assert gs.T_final == os_.T_final
    assert list(gs.w_repair) == list(os_.w_repair)
    assert list(gs.w_destroy) == list(os_.w_destroy)
    assert np.array_equal(g["best_ops"], o["best_ops"]) and np.array_equal(g["best_off"], o["best_off"])
    assert np.array_equal(g["cur_ops"], o["cur_ops"]) and np.array_equal(g["cur_off"], o["cur_off"])
    # every returned solution re-evaluated by the oracle
    assert oracle.evaluate(oi, g["best_ops"], g["best_off"]) == (g["z_best"], 0)
    assert oracle.evaluate(oi, g["cur_ops"], g["cur_off"]) == (g["z_current"], 0)


def test_alns_n16_trajectory(vrp):
    # the tiny workload: n=16, m=2, R=4, Q=4, base p; 200 iterations from seed 0
    cfg = workloads.CONFIGS["tiny_n16"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], seed=0)
    _, oi, g, o = run_both(vrp, w, 200, seed=0)
    assert_same_run(oi, g, o)
    assert g["z_best"] <= g["trace"][0]


@pytest.mark.parametrize("mask", [1, 2, 4, 8, 15])
def test_alns_single_repair_operator(vrp, mask):
    w = workloads.make_instance(24, 3, 6, 4, "5x", seed=3)
    _, oi, g, o = run_both(vrp, w, 60, seed=7, mask=mask)
    assert_same_run(oi, g, o)


def test_alns_medium_trajectory(vrp):
    # the n=100 ALNS workload's shape (m=4, R=10, Q=5, 2x, q = 10% of n) at n=40 so the
    # oracle's full re-simulation stays quick
    w = workloads.make_instance(40, 4, 10, 5, "2x", seed=2)
    _, oi, g, o = run_both(vrp, w, 6, seed=1, q=(4, 4))
    assert_same_run(oi, g, o)


def test_alns_team_blocks_agree(vrp):
    w = workloads.make_instance(100, 4, 10, 5, "2x", seed=0)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(oi, w.coords)
    runs = [vrp.alns_run(inst, vrp.alns_params(8, 10, 10, 3, tb), seed=3, init=init) for tb in (1, 6)]
    assert runs[1]["stats"].team_blocks == 6
    assert np.array_equal(runs[0]["trace"], runs[1]["trace"])
    assert np.array_equal(runs[0]["best_ops"], runs[1]["best_ops"])
    assert oracle.evaluate(oi, runs[0]["best_ops"], runs[0]["best_off"]) == (runs[0]["z_best"], 0)


def test_alns_n1000_reevaluated(vrp):
    cfg = workloads.CONFIGS["serving_n1000"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=0)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    g = vrp.alns_run(inst, vrp.alns_params(3), seed=0)
    assert oracle.evaluate(oi, g["best_ops"], g["best_off"]) == (g["z_best"], 0)
    assert oracle.evaluate(oi, g["cur_ops"], g["cur_off"]) == (g["z_current"], 0)
    assert g["stats"].matrix_entries > 0


def test_matrix_n1000_sampled(vrp):
    cfg = workloads.CONFIGS["serving_n1000"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=1)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops, off = vrp.initial_solution(inst)
    rng = np.random.default_rng(0)
    remove = rng.choice(np.arange(1, w.n + 1), size=30, replace=False)
    po, pf = destroyed(ops, off, w.m, remove)
    c = int(remove[0])
    dg, tg = vrp.insertion_matrix(inst, po, pf, c)
    z0, st0 = oracle.evaluate(oi, po, pf, allow_partial=True)
    G = dg.shape[0]
    gaps = [(v, i) for v in range(w.m) for i in range(pf[v + 1] - pf[v] + 1)]
    idx = rng.choice(G * G, size=300, replace=False)
    for flat in idx:
        r, col = divmod(int(flat), G)
        (a, i), (b, j) = gaps[r], gaps[col]
        if a == b and j < i:
            assert dg[r, col] == INT32_MAX
            continue
        routes = [list(po[pf[v]:pf[v + 1]]) for v in range(w.m)]
        if a == b:
            routes[a] = routes[a][:i] + [2 * c] + routes[a][i:j] + [2 * c + 1] + routes[a][j:]
        else:
            routes[a] = routes[a][:i] + [2 * c] + routes[a][i:]
            routes[b] = routes[b][:j] + [2 * c + 1] + routes[b][j:]
        so = np.array(sum(routes, []), np.int32)
        sf = np.zeros(w.m + 1, np.int32)
        sf[1:] = np.cumsum([len(x) for x in routes])
        z, st = oracle.evaluate(oi, so, sf, allow_partial=True)
        cap = any(_route_cap_bad(routes[v], w.Q) for v in {a, b})
        expect = INT32_MAX if (st & (oracle.CYCLE | oracle.POOL)) or cap else z - z0
        assert dg[r, col] == expect, (r, col, dg[r, col], expect)


def _route_cap_bad(route, Q):
    s = smin = smax = 0
    for o in route:
        s += 1 if o & 1 else -1
        smin, smax = min(smin, s), max(smax, s)
    return -smin + smax > Q


def test_alns_all_repair_operators_medium(vrp):
    # greedy, regret-2, regret-3 and regret-m drawn by the roulette (Section 4.2.3)
    w = workloads.make_instance(40, 5, 10, 5, "2x", seed=5)
    _, oi, g, o = run_both(vrp, w, 8, seed=2, q=(4, 4), mask=15)
    assert_same_run(oi, g, o)


@pytest.mark.parametrize("dmask", [1, 2, 4, 8, 16, 32, 63])
def test_alns_destroy_operators(vrp, dmask):
    # random, worst, Shaw, cluster, route and critical-path removal alone,
    # then all six under the roulette (Section 4.2.2)
    w = workloads.make_instance(24, 3, 6, 4, "5x", seed=4)
    _, oi, g, o = run_both(vrp, w, 60, seed=11, dmask=dmask)
    assert_same_run(oi, g, o)


@pytest.mark.parametrize("seed", range(2))
def test_alns_all_operators_medium(vrp, seed):
    # every destroy and repair operator, a removal range wide enough for the
    # route and critical-path top-ups, clustered coordinates
    w = workloads.make_instance(40, 5, 10, 5, "2x", "clustered", seed=8 + seed)
    _, oi, g, o = run_both(vrp, w, 24, seed=seed, q=(3, 8), mask=15, dmask=63)
    assert_same_run(oi, g, o)


def test_alns_all_operators_team_blocks_agree(vrp):
    w = workloads.make_instance(100, 4, 10, 5, "2x", seed=1)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(oi, w.coords)
    runs = [vrp.alns_run(inst, vrp.alns_params(12, 5, 15, 15, tb, destroy_mask=63), seed=5, init=init)
            for tb in (1, 7)]
    assert np.array_equal(runs[0]["trace"], runs[1]["trace"])
    assert np.array_equal(runs[0]["best_ops"], runs[1]["best_ops"])
    assert list(runs[0]["stats"].w_destroy) == list(runs[1]["stats"].w_destroy)
    assert oracle.evaluate(oi, runs[0]["best_ops"], runs[0]["best_off"]) == (runs[0]["z_best"], 0)


@pytest.mark.parametrize("ls", [(3, 0), (0, 4), (3, 5)])
def test_alns_local_search(vrp, ls):
    # pickup repositioning and cross-agent relocation (Section 4.2.6) at short
    # periods so that they run many times
    w = workloads.make_instance(24, 3, 6, 4, "5x", seed=6)
    _, oi, g, o = run_both(vrp, w, 45, seed=3, ls=ls)
    assert_same_run(oi, g, o)
    assert g["stats"].ls_moves > 0


@pytest.mark.parametrize("seed", range(2))
def test_alns_local_search_all_operators_medium(vrp, seed):
    w = workloads.make_instance(40, 5, 10, 5, "2x", "clustered", seed=20 + seed)
    _, oi, g, o = run_both(vrp, w, 20, seed=seed, q=(3, 8), mask=15, dmask=63, ls=(4, 6))
    assert_same_run(oi, g, o)


def test_alns_local_search_load_full_tight(vrp):
    # the paper's fleet with every vehicle leaving full: capacity binds, so
    # removing a customer can leave its old route infeasible
    w = workloads.make_paper_instance(30, "1R20", seed=4)
    _, oi, g, o = run_both(vrp, w, 30, seed=1, q=(3, 6), dmask=63, ls=(2, 3), load_full=True)
    assert_same_run(oi, g, o)


def test_alns_local_search_team_blocks_agree(vrp):
    w = workloads.make_instance(100, 4, 10, 5, "2x", seed=2)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(oi, w.coords)
    runs = [vrp.alns_run(inst, vrp.alns_params(10, 5, 10, 3, tb, ls_pickup_every=3, ls_relocate_every=5),
                         seed=4, init=init) for tb in (1, 9)]
    assert np.array_equal(runs[0]["trace"], runs[1]["trace"])
    assert np.array_equal(runs[0]["best_ops"], runs[1]["best_ops"])
    assert runs[0]["stats"].ls_moves == runs[1]["stats"].ls_moves
    assert oracle.evaluate(oi, runs[0]["best_ops"], runs[0]["best_off"]) == (runs[0]["z_best"], 0)


def replicas_both(vrp, w, iters, seed, R, sync, q=(0, 0), mask=3, dmask=1, ls=(200, 500), team_blocks=0):
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    init = oracle.initial_solution(oi, w.coords)
    g = vrp.alns_run(inst, vrp.alns_params(iters, q[0], q[1], mask, team_blocks, destroy_mask=dmask,
                                           ls_pickup_every=ls[0], ls_relocate_every=ls[1], replicas=R,
                                           sync_every=sync), seed=seed, init=init)
    o = oracle.alns_run_replicas(oi, init[0], init[1],
                                 oracle.alns_params(iters, q[0], q[1], mask, destroy_mask=dmask,
                                                    ls_pickup_every=ls[0], ls_relocate_every=ls[1]),
                                 seed, R, sync)
    assert np.array_equal(g["traces"], o["traces"]), np.argwhere(g["traces"] != o["traces"])[:5]
    gs = g["stats"]
    assert gs.replicas == R and gs.imports == o["imports"] and gs.best_replica == o["best_replica"]
    for f in ("accepted", "improved", "new_best", "reheats", "rejected_infeasible", "ls_moves"):
        assert getattr(gs, f) == sum(getattr(st, f) for st in o["stats"]), f
    assert np.array_equal(g["best_ops"], o["best_ops"]) and np.array_equal(g["best_off"], o["best_off"])
    assert oracle.evaluate(oi, g["best_ops"], g["best_off"]) == (g["z_best"], 0)
    return g, o


@pytest.mark.parametrize("R,sync", [(3, 5), (4, 7)])
def test_alns_replicas_small(vrp, R, sync):
    # multi-instance ALNS (Section 4.2.1): replicas on their own streams, the
    # best of all imported at every checkpoint
    w = workloads.make_instance(24, 3, 6, 4, "5x", seed=7)
    g, o = replicas_both(vrp, w, 30, 5, R, sync, q=(3, 6), mask=15, dmask=63, ls=(9, 13))
    assert o["imports"] > 0


def test_alns_replicas_medium(vrp):
    # several CTAs per replica (the grid barrier spans teams of 8)
    w = workloads.make_instance(60, 4, 10, 5, "2x", seed=3)
    g, o = replicas_both(vrp, w, 8, 5, 4, 3, q=(4, 8))
    assert g["stats"].team_blocks > 1


@pytest.mark.parametrize("n,m,R,Q,v,lay", [(16, 2, 4, 4, "base", "uniform"), (40, 4, 10, 5, "2x", "uniform"),
                                           (60, 5, 20, 4, "1R20", "clustered"), (7, 5, 3, 2, "base", "uniform"),
                                           (1000, 20, 100, 10, "1R20", "mixed")])
def test_initial_solution_paper_matches_oracle(vrp, n, m, R, Q, v, lay):
    # the three-phase constructor alone (Section 4.2.5)
    w = workloads.make_instance(n, m, R, Q, v, lay, seed=n)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    go, gf, gz = vrp.initial_solution_paper(inst, 0)
    oo, of = oracle.initial_solution_paper(oi, w.coords, 0)
    assert np.array_equal(go, oo) and np.array_equal(gf, of)
    assert oracle.evaluate(oi, go, gf) == (gz, 0)


@pytest.mark.parametrize("n,m,R,Q,v", [(24, 3, 8, 4, "5x"), (40, 5, 10, 5, "2x")])
def test_initial_solution_paper_refined_matches_oracle(vrp, n, m, R, Q, v):
    w = workloads.make_instance(n, m, R, Q, v, seed=n + 1)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    go, gf, gz = vrp.initial_solution_paper(inst, 10)
    oo, of = oracle.initial_solution_paper(oi, w.coords, 10)
    assert np.array_equal(go, oo) and np.array_equal(gf, of)
    assert oracle.evaluate(oi, go, gf) == (gz, 0)


def test_alns_from_the_paper_start(vrp):
    w = workloads.make_instance(24, 3, 8, 4, "2x", seed=12)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    g = vrp.alns_run(inst, vrp.alns_params(30, init_mode=1), seed=4)
    init = oracle.initial_solution_paper(oi, w.coords, 10)
    o = oracle.alns_run(oi, init[0], init[1], oracle.alns_params(30), 4)
    assert np.array_equal(g["trace"], o["trace"]) and g["stats"].z_init == o["stats"].z_init
    assert np.array_equal(g["best_ops"], o["best_ops"])


@pytest.mark.parametrize("mask", [3, 2, 4])
def test_alns_c3_shape_many_ctas(vrp, mask):
    """The BRKGA workload's instance (n=200, 8 Gaussian clusters, m=6, R=20,
    Q=6, 5x) searched by a team of 64 CTAs for two iterations, replayed by the
    oracle: the incremental longest-path updates and the shortcut-gap entries
    both run (Section 4.2.3), and the tiles' lower bounds leave entries and
    whole tiles unscored, under greedy with regret-2 (the bench's operators),
    regret-2 alone and regret-3 alone: each repair rule's bound is exercised
    against the oracle's full matrices."""
    cfg = workloads.CONFIGS["brkga_n200"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=0)
    # draw seed 3 removes customers with shortcut gaps in these two iterations
    _, oi, g, o = run_both(vrp, w, 2, seed=3, q=(5, 5), mask=mask, team_blocks=64)
    st = g["stats"]
    assert st.team_blocks == 64
    assert_same_run(oi, g, o)
    assert st.pruned_entries > 0 and st.tiles_pruned > 0
    if mask == 3:
        assert st.incremental_steps > 0 and st.full_steps > 0
        assert st.fallback_entries > 0


def _shortcut_gaps(d, ops, off, m, c):
    """Gaps (x, y) of the partial solution where the rounded legs through c are
    shorter than x -> y: there the tile formula does not hold and the entries
    come from the shortcut simulations."""
    n_sc = 0
    for v in range(m):
        r = [0] + [o >> 1 for o in ops[off[v]:off[v + 1]]] + [0]
        for x, y in zip(r[:-1], r[1:]):
            n_sc += int(d[x, c]) + int(d[c, y]) < int(d[x, y])
    return n_sc


def test_repair_steps_then_matrix_c3_shortcuts(vrp):
    """n = 200 clustered (m=6, R=20, Q=6, 5x) on 64 CTAs: removed customers
    chosen so that shortcut gaps occur; each of four repair steps equals the
    oracle's and each next matrix equals its full re-simulation."""
    cfg = workloads.CONFIGS["brkga_n200"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=2)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops, off = oracle.initial_solution(oi, w.coords)
    rng = np.random.default_rng(0)
    for _ in range(500):
        removed = sorted(rng.choice(np.arange(1, w.n + 1), size=5, replace=False).tolist())
        po, pf = _partial(ops, off, w.m, removed)
        if _shortcut_gaps(oi.d, po, pf, w.m, removed[0]) > 0:
            break
    else:
        pytest.fail("no removal with a shortcut gap")
    seen_sc = 0
    incr_total = 0
    for steps in range(4):
        go, gf, dg, tg, incr = vrp.repair_then_matrix(inst, po, pf, removed, steps, team_blocks=64)
        oo, of = oracle.repair(oi, 0, po, pf, removed, max_steps=steps)
        assert np.array_equal(gf, of) and np.array_equal(go, oo), steps
        left = [c for c in removed if 2 * c not in set(go.tolist())]
        seen_sc += _shortcut_gaps(oi.d, go, gf, w.m, left[0])
        md, mt, _ = oracle.insertion_matrix(oi, go, gf, left[0])
        assert np.array_equal(dg, md), steps
        ok = md != INT32_MAX
        assert np.array_equal(tg[ok], mt[ok]), steps
        incr_total += incr
    assert seen_sc > 0 and incr_total > 0


def _partial(ops, off, m, removed):
    rem = set(int(c) for c in removed)
    routes = [[o for o in ops[off[v]:off[v + 1]] if (o >> 1) not in rem] for v in range(m)]
    po = np.array([o for r in routes for o in r], np.int32)
    pf = np.zeros(m + 1, np.int32)
    pf[1:] = np.cumsum([len(r) for r in routes])
    return po, pf


@pytest.mark.parametrize("op", [0, 1])
def test_repair_steps_then_matrix_small(vrp, op):
    """Part of a repair on the device, then the next matrix: the steps equal
    the oracle's repair steps, and the whole matrix (after incremental
    longest-path updates) equals the oracle's full re-simulation."""
    w = workloads.make_instance(40, 4, 10, 5, "2x", seed=8)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops, off = oracle.initial_solution(oi, w.coords)
    removed = sorted(np.random.default_rng(3).choice(np.arange(1, 41), size=6, replace=False).tolist())
    po, pf = _partial(ops, off, w.m, removed)
    incr_total = 0
    for steps in range(0, 6):
        go, gf, dg, tg, incr = vrp.repair_then_matrix(inst, po, pf, removed, steps, repair_op=op, team_blocks=3)
        oo, of = oracle.repair(oi, op, po, pf, removed, max_steps=steps)
        assert np.array_equal(gf, of) and np.array_equal(go, oo), steps
        left = [c for c in removed if 2 * c not in set(go.tolist())]
        md, mt, _ = oracle.insertion_matrix(oi, go, gf, left[0])
        assert np.array_equal(dg, md), steps
        ok = md != INT32_MAX
        assert np.array_equal(tg[ok], mt[ok]), steps
        incr_total += incr
    assert incr_total > 0


def test_repair_steps_then_matrix_n1000(vrp):
    """At n = 1000 (m=20, R=100, Q=10, 1R20) on the whole GPU: eight greedy
    steps from the three-phase start with 30 customers removed, most of them
    incremental, then 400 sampled entries of the next matrix against the
    oracle's re-simulation of the partial solution the steps produced."""
    cfg = workloads.CONFIGS["serving_n1000"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=2)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    ops, off, _ = vrp.initial_solution_paper(inst, refine_rounds=0)
    rng = np.random.default_rng(5)
    removed = sorted(rng.choice(np.arange(1, w.n + 1), size=30, replace=False).tolist())
    po, pf = _partial(ops, off, w.m, removed)
    steps = 8
    go, gf, dg, tg, incr = vrp.repair_then_matrix(inst, po, pf, removed, steps)
    assert incr >= 5, incr
    # the steps inserted eight whole customers into the partial solution and moved nothing else
    present = set(go.tolist())
    inserted = [c for c in removed if 2 * c in present]
    assert len(inserted) == steps and all(2 * c + 1 in present for c in inserted)
    keep = set(inserted)
    assert np.array_equal(_partial(go, gf, w.m, keep)[0], po)
    assert oracle.evaluate(oi, go, gf, allow_partial=True)[1] & (oracle.CYCLE | oracle.MALFORMED) == 0
    c = [x for x in removed if x not in keep][0]
    z0, _ = oracle.evaluate(oi, go, gf, allow_partial=True)
    G = dg.shape[0]
    gaps = [(v, i) for v in range(w.m) for i in range(gf[v + 1] - gf[v] + 1)]
    for flat in rng.choice(G * G, size=400, replace=False):
        r, col = divmod(int(flat), G)
        (a, i), (b, j) = gaps[r], gaps[col]
        if a == b and j < i:
            assert dg[r, col] == INT32_MAX
            continue
        routes = [list(go[gf[v]:gf[v + 1]]) for v in range(w.m)]
        if a == b:
            routes[a] = routes[a][:i] + [2 * c] + routes[a][i:j] + [2 * c + 1] + routes[a][j:]
        else:
            routes[a] = routes[a][:i] + [2 * c] + routes[a][i:]
            routes[b] = routes[b][:j] + [2 * c + 1] + routes[b][j:]
        so = np.array(sum(routes, []), np.int32)
        sf = np.zeros(w.m + 1, np.int32)
        sf[1:] = np.cumsum([len(x) for x in routes])
        z, st = oracle.evaluate(oi, so, sf, allow_partial=True)
        cap = any(_route_cap_bad(routes[v], w.Q) for v in {a, b})
        expect = INT32_MAX if (st & (oracle.CYCLE | oracle.POOL)) or cap else z - z0
        assert dg[r, col] == expect, (r, col, dg[r, col], expect)
