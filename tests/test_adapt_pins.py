"""Pins of Algorithm 1's acceptance and adaptation (Section 4.2.4, Table 2) in
the oracle, on scripted iterations whose outcome is worked out by hand below:
scores sigma = (33, 9, 13) for a new best, an improving and an accepted
worse candidate; no score for a rejection; an equal makespan goes to the SA
test with exp(0) = 1 (always accepted); the weight update
w <- max(w_min, (1 - r) w + r s/a) every tau iterations with s/a = 0 for an
operator without attempts; cooling T <- alpha T from T0 z_init; the reheat
T <- reheat T0 z_best only once the stagnation count is reached AND T is
below 1% of its start, the count restarting on a new best only."""
import pytest

import oracle

CAP = 2          # VEH_CAP status bit


def params(**kw):
    P = oracle.alns_params(0)
    for k, v in kw.items():
        setattr(P, k, v)
    return P


def close(a, b):
    return abs(a - b) <= 1e-12 * max(1.0, abs(b))


def test_scores_and_weights_hand_trace():
    # z0 = 1000, T0 = 0.3: T starts at 300.  Iterations (destroy, repair, z', status, u):
    steps = [
        (0, 0, 900, 0, 0.5),        # 1: below the best -> new best, sigma1 = 33 to d0 and r0
        (1, 1, 950, 0, 0.0),        # 2: worse by 50, u = 0 < exp(-50/T) -> accepted, sigma3 = 13 to d1, r1
        (0, 2, 920, 0, 0.9),        # 3: below current 950, above best 900 -> sigma2 = 9 to d0, r2
        (1, 0, 800, CAP, 0.0),      # 4: a status bit -> rejected, no score
        (0, 0, 990, 0, 0.99),       # 5: worse by 70, exp(-70/299.76) = 0.79 < 0.99 -> rejected
        (2, 0, 920, 0, 0.999999),   # 6: equal -> exp(0) = 1 > u -> accepted, sigma3 = 13 to d2, r0
    ]
    P = params(tau=6)
    st, trace = oracle.alns_adapt_script(P, 1000, steps)
    assert list(trace) == [900, 950, 920, 920, 920, 920]
    assert (st.accepted, st.improved, st.new_best, st.rejected_infeasible, st.reheats) == (4, 2, 1, 1, 0)
    assert (st.z_best, st.z_current, st.z_init) == (900, 920, 1000)
    # weights at iteration 6, w = 0.9 * 1 + 0.1 * s/a:
    #   destroy 0: a = 3 (it 1, 3, 5), s = 33 + 9 = 42  -> 0.9 + 1.4  = 2.3
    #   destroy 1: a = 2 (it 2, 4),    s = 13           -> 0.9 + 0.65 = 1.55
    #   destroy 2: a = 1 (it 6),       s = 13           -> 0.9 + 1.3  = 2.2
    #   destroy 3-5: no attempts                        -> 0.9
    #   repair 0: a = 4 (it 1, 4, 5, 6), s = 33 + 13 = 46 -> 0.9 + 1.15 = 2.05
    #   repair 1: a = 1 (it 2), s = 13 -> 2.2;  repair 2: a = 1 (it 3), s = 9 -> 1.8;  repair 3 -> 0.9
    for got, want in zip(st.w_destroy[:6], [2.3, 1.55, 2.2, 0.9, 0.9, 0.9]):
        assert close(got, want), list(st.w_destroy)
    for got, want in zip(st.w_repair, [2.05, 2.2, 1.8, 0.9]):
        assert close(got, want), list(st.w_repair)
    assert close(st.T_final, 300.0 * 0.9998 ** 6)


def test_weights_before_tau_and_the_floor():
    steps = [(0, 0, 900, 0, 0.5), (1, 1, 950, 0, 0.0)]
    st, _ = oracle.alns_adapt_script(params(tau=3), 1000, steps)
    assert list(st.w_destroy[:6]) == [1.0] * 6 and list(st.w_repair) == [1.0] * 4      # no update yet
    # r = 0.95: an operator with a = 0 or s = 0 falls to 0.05 and is floored at w_min = 0.1;
    # destroy 1 / repair 1 accepted a worse candidate: 0.05 + 0.95 * 13 = 12.4
    st, _ = oracle.alns_adapt_script(params(tau=2, r=0.95), 1000, [(0, 0, 1000, CAP, 0.5), (1, 1, 1010, 0, 0.0)])
    assert close(st.w_destroy[0], 0.1) and close(st.w_destroy[1], 12.4) and close(st.w_destroy[2], 0.1)
    assert close(st.w_repair[0], 0.1) and close(st.w_repair[1], 12.4) and close(st.w_repair[3], 0.1)


def test_reheat_needs_the_temperature_gate():
    # alpha = 0.05: T = 300 -> 15 -> 0.75 (< 1% of 300 = 3) with stagnation 2 after it 2
    steps = [(0, 0, 900, 0, 0.5), (0, 0, 1000, 0, 0.999), (0, 0, 1000, 0, 0.999)]
    st, trace = oracle.alns_adapt_script(params(alpha=0.05, stagnation=2), 1000, steps)
    assert st.reheats == 1 and list(trace) == [900, 900, 900]
    # reheat at it 2: T = 0.5 * 0.3 * z_best 900 = 135, then one more cooling step
    assert close(st.T_final, (0.5 * 0.3) * 900.0 * 0.05)
    # alpha = 0.9: T = 270, 243, 218.7 never falls below 3 -> no reheat although stagnation is reached
    st, _ = oracle.alns_adapt_script(params(alpha=0.9, stagnation=2), 1000, steps)
    assert st.reheats == 0 and close(st.T_final, 300.0 * 0.9 ** 3)
    # the gate is open but the stagnation count (5) is not reached
    st, _ = oracle.alns_adapt_script(params(alpha=0.05, stagnation=5), 1000, steps)
    assert st.reheats == 0


def test_stagnation_restarts_only_on_a_new_best():
    # it 1: worse, accepted (u = 0); it 2: improving but not below the best 1000.
    # The count reaches 2 and T = 0.75 < 3: reheat to 0.15 * z_best 1000 = 150
    steps = [(0, 0, 1100, 0, 0.0), (0, 0, 1050, 0, 0.5)]
    st, trace = oracle.alns_adapt_script(params(alpha=0.05, stagnation=2), 1000, steps)
    assert list(trace) == [1100, 1050] and st.improved == 1 and st.new_best == 0
    assert st.reheats == 1 and close(st.T_final, (0.5 * 0.3) * 1000.0)
    # with a new best at it 2 instead the count restarts and nothing reheats
    st, _ = oracle.alns_adapt_script(params(alpha=0.05, stagnation=2), 1000, [(0, 0, 1100, 0, 0.0),
                                                                              (0, 0, 990, 0, 0.5)])
    assert st.reheats == 0 and st.new_best == 1


@pytest.mark.parametrize("delta,u,accept", [(50, 0.846, True), (50, 0.847, False), (1, 0.9966, True),
                                            (1, 0.9967, False)])
def test_sa_threshold(delta, u, accept):
    # T = 300 at the first iteration: exp(-50/300) = 0.84648, exp(-1/300) = 0.996672
    st, trace = oracle.alns_adapt_script(params(), 1000, [(0, 0, 1000 + delta, 0, u)])
    assert (st.accepted == 1) == accept and trace[0] == (1000 + delta if accept else 1000)
