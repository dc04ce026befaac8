"""Continuous-batching server: requests of different n arrive while others run,
are admitted by memory budget, overlap on the device, and each answer equals
the one the same request gets alone; every answer re-evaluated by the oracle."""
import time

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def requests():
    out = []
    for i, n in enumerate([20, 60, 35, 90, 16, 75, 50, 28]):
        m = 2 + i % 3
        out.append(workloads.make_instance(n, m, R=max(m, n // 8), Q=4, variant="2x", seed=50 + i))
    return out


def test_mix_equals_alone(vrp):
    ws = requests()
    srv = vrp.Server(mem_budget_bytes=8 << 30, max_active=4)
    ids = []
    rng = np.random.default_rng(0)
    for i, w in enumerate(ws):
        ids.append(srv.submit(w, alns_iterations=30, brkga_pop=64, brkga_generations=8, seed=i))
        time.sleep(float(rng.exponential(0.01)))          # Poisson-like arrivals
    mixed = [srv.wait(r) for r in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(ws) and st["peak_active"] >= 2
    alone = []
    for i, w in enumerate(ws):
        s1 = vrp.Server(mem_budget_bytes=8 << 30, max_active=1)
        alone.append(s1.wait(s1.submit(w, alns_iterations=30, brkga_pop=64, brkga_generations=8, seed=i)))
        s1.close()
    for w, a, b in zip(ws, mixed, alone):
        assert a["status"] == 0 and b["status"] == 0, (a["message"], b["message"])
        assert (a["z_alns"], a["z_brkga"], a["z_best"]) == (b["z_alns"], b["z_brkga"], b["z_best"])
        assert np.array_equal(a["ops"], b["ops"]) and np.array_equal(a["off"], b["off"])
        oi = oracle.OracleInstance.from_workload(w)
        assert oracle.evaluate(oi, a["ops"], a["off"]) == (a["z_best"], 0)


def test_admission_by_memory(vrp):
    ws = requests()[:4]
    # a budget too small for two requests at once: they run one after another
    srv = vrp.Server(mem_budget_bytes=3 << 20, max_active=4)
    ids = [srv.submit(w, alns_iterations=5, seed=i) for i, w in enumerate(ws)]
    res = [srv.wait(r) for r in ids]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    assert st["peak_bytes"] <= 3 << 20
    big = workloads.make_instance(1000, 20, 100, 10, seed=1)
    srv = vrp.Server(mem_budget_bytes=1 << 20, max_active=1)
    with pytest.raises(vrp.VrpError):
        srv.submit(big, alns_iterations=5)
    srv.close()


def test_withdraw_pending(vrp):
    """A bounded serving window withdraws the requests not admitted yet: they
    complete at once with EBUSY (-5) and no latency sample, while the admitted
    one finishes and is re-evaluated by the oracle."""
    ws = requests()[:5]
    srv = vrp.Server(mem_budget_bytes=8 << 30, max_active=1)
    ids = [srv.submit(w, alns_iterations=200, seed=i) for i, w in enumerate(ws)]
    time.sleep(0.05)
    k = srv.cancel_pending()
    res = [srv.wait(r) for r in ids]
    st = srv.stats()
    srv.close()
    ran = [r for r in res if r["status"] == 0]
    gone = [r for r in res if r["status"] != 0]
    assert k == len(gone) and k >= 1 and len(ran) >= 1
    assert all(r["status"] == -5 and "withdrawn" in r["message"] for r in gone)
    assert st["completed"] == len(ran)
    for w, r in zip(ws, res):
        if r["status"] == 0:
            oi = oracle.OracleInstance.from_workload(w)
            assert oracle.evaluate(oi, r["ops"], r["off"]) == (r["z_best"], 0)
