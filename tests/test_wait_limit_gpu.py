"""Failure detection of the ALNS team's device-side waits.

Every spin-wait of the team (its barriers, and the wait for the shortcut
simulations) gives up after a limit, records the error and lets the kernel
return, so a lost CTA ends the run with VRPRPD_ETIMEOUT instead of hanging
the GPU.  The test makes the waits run out without any fault: with a limit
of 1 ns every CTA that is not the last to arrive at the first team barrier
gives up at once.  The run must report VRPRPD_ETIMEOUT, and the library and
the CUDA context must stay usable: the same instance then runs normally and
its result is re-evaluated by the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

VRPRPD_ETIMEOUT = -4


def test_alns_wait_that_runs_out_reports_timeout(vrp):
    w = workloads.make_instance(200, 6, 20, 6, "5x", "clustered", seed=0)
    inst = vrp.Instance.from_workload(w)
    p = vrp.alns_params(3, team_blocks=16, wait_limit_ns=1)
    with pytest.raises(vrp.VrpError) as err:
        vrp.alns_run(inst, p, seed=0)
    assert err.value.code == VRPRPD_ETIMEOUT
    assert "timed out" in str(err.value)
    # the same library, instance and context afterwards
    r = vrp.alns_run(inst, vrp.alns_params(3, team_blocks=16), seed=0)
    oi = oracle.OracleInstance.from_workload(w)
    ops = np.asarray(r["best_ops"], np.int32)[None, :]
    off = np.asarray(r["best_off"], np.int32)[None, :]
    z, st = oracle.evaluate_batch(oi, ops, off)
    assert int(st[0]) == 0 and int(z[0]) == r["z_best"]
