"""Many instances of uneven size in one persistent launch (the uneven-instance
workload's shape: n log-uniform in [17, 500]): every candidate bit-exact against the oracle and against the
one-launch-per-instance plain form; graph replay gives the same results."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_uneven_instances_one_launch(vrp):
    import torch
    insts = workloads.uneven_instances(24, 17, 500, 8, "1R10", seed=3)
    items, host = [], []
    rng = np.random.default_rng(0)
    for i, w in enumerate(insts):
        cnt = int(rng.integers(1, 300))
        if i % 2:
            ops, off = workloads.precedence_candidates(w.n, w.m, cnt, seed=i)
        else:
            ops, off = workloads.random_candidates(w.n, w.m, cnt, seed=i)
        inst = vrp.Instance.from_workload(w)
        items.append((inst, torch.from_numpy(ops).cuda(), torch.from_numpy(off).cuda()))
        host.append((w, ops, off))
    mb = vrp.MultiBatch(items)
    expect = [oracle.evaluate_batch(oracle.OracleInstance.from_workload(w), ops, off, threads=8)
              for w, ops, off in host]
    z, st = mb.evaluate()
    torch.cuda.synchronize()
    for (zo, so), zi, si, (inst, dops, doff) in zip(expect, z, st, items):
        assert np.array_equal(zi.cpu().numpy(), zo)
        assert np.array_equal(si.cpu().numpy().astype(np.uint32), so)
        zp, sp = vrp.evaluate_plain(inst, dops, doff)
        assert np.array_equal(zp.cpu().numpy(), zo)
    # both walks by hand, both distance modes
    for walk in ("staged", "streamed"):
        for mode in ("global16", "global32"):
            mb.set_config(mode, 8, walk)
            zz, ss = mb.evaluate()
            torch.cuda.synchronize()
            for (zo, so), zi, si in zip(expect, zz, ss):
                assert np.array_equal(zi.cpu().numpy(), zo), (walk, mode)
                assert np.array_equal(si.cpu().numpy().astype(np.uint32), so), (walk, mode)
            z = [t.clone() for t in zz]
    cfg = mb.autotune()
    assert cfg["warps_per_block"] > 0
    z2, st2 = mb.evaluate()                     # replayed graph after re-planning
    mb.evaluate()
    torch.cuda.synchronize()
    for a, b in zip(z, z2):
        assert torch.equal(a, b)
