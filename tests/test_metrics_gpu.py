"""GPU parity of the Section 5.2 coordination counts (Cross-Agent and
Interleaved) against the oracle: bit-exact per candidate on precedence-
consistent candidates (every schedule exists), random candidates (mostly
cyclic: interleaved undefined), ALNS solutions, malformed candidates, m = 1
and m = 32, ragged batches, and a sampled check at n = 1000."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def both(vrp, w, ops, off, sample=None):
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    cr, il = vrp.coordination(inst, dev(ops), dev(off))
    cr, il = cr.cpu().numpy(), il.cpu().numpy()
    idx = range(len(ops)) if sample is None else sample
    for k in idx:
        c, i, _ = oracle.coordination(oi, ops[k], off[k])
        assert (cr[k], il[k]) == (c, i), (k, cr[k], il[k], c, i)
    return cr, il


@pytest.mark.parametrize("n,m,variant", [(16, 2, "base"), (37, 5, "5x"), (100, 4, "2x"), (61, 32, "1R20"),
                                         (25, 1, "5x")])
def test_precedence_candidates(vrp, n, m, variant):
    w = workloads.make_instance(n, m, n, 8, variant, seed=n + m)
    ops, off = workloads.precedence_candidates(n, m, 301, seed=n)
    cr, il = both(vrp, w, ops, off)
    assert (il >= 0).all()
    if m == 1:
        assert (cr == 0).all()


@pytest.mark.parametrize("n,m", [(12, 3), (40, 6)])
def test_random_candidates_with_cycles(vrp, n, m):
    w = workloads.make_instance(n, m, n, 8, "2x", seed=3)
    ops, off = workloads.random_candidates(n, m, 257, seed=4)
    cr, il = both(vrp, w, ops, off)
    assert (il == -1).any() and (cr >= 0).all()


def test_distance_paths_agree(vrp):
    # legs recomputed from small coordinates, gathered from the matrix of an
    # instance built from d, and gathered for coordinates too spread for the
    # fp32 path: the same counts as the oracle
    n, m = 50, 4
    w = workloads.make_instance(n, m, n, 8, "2x", seed=11)
    ops, off = workloads.precedence_candidates(n, m, 200, seed=11)
    rops, roff = workloads.random_candidates(n, m, 100, seed=12)
    ops, off = np.concatenate([ops, rops]), np.concatenate([off, roff])
    cr, il = both(vrp, w, ops, off)
    inst_d = vrp.Instance(m, n, 8, w.p, d=oracle.euc2d(w.coords))
    c2, i2 = vrp.coordination(inst_d, dev(ops), dev(off))
    assert np.array_equal(c2.cpu().numpy(), cr) and np.array_equal(i2.cpu().numpy(), il)
    both(vrp, workloads.Instance(w.coords * 40, w.p, m, n, 8), ops, off)


def test_malformed(vrp):
    n, m = 10, 3
    w = workloads.make_instance(n, m, n, 8, "base", seed=1)
    ops, off = workloads.precedence_candidates(n, m, 6, seed=1)
    ops, off = ops.copy(), off.copy()
    ops[0, 3] = ops[0, 4]            # duplicate op
    ops[1, 0] = 2 * n + 2            # out of range
    ops[2, 5] = 1                    # depot code
    off[3, 1] = off[3, 2] + 1        # offsets decrease
    off[4, m] = 2 * n - 1            # offsets end short
    cr, il = both(vrp, w, ops, off)
    assert list(cr[:5]) == [-1] * 5 and list(il[:5]) == [-1] * 5 and cr[5] >= 0


def test_alns_solutions(vrp):
    w = workloads.make_instance(60, 4, 10, 5, "5x", seed=2)
    inst = vrp.Instance.from_workload(w)
    sols = []
    for seed in range(4):
        g = vrp.alns_run(inst, vrp.alns_params(40, destroy_mask=63, repair_mask=15), seed=seed)
        sols += [(g["best_ops"], g["best_off"]), (g["cur_ops"], g["cur_off"])]
    ops = np.stack([s[0] for s in sols]).astype(np.int32)
    off = np.stack([s[1] for s in sols]).astype(np.int32)
    cr, il = both(vrp, w, ops, off)
    assert (il >= 0).all()


def test_n1000_sampled(vrp):
    w = workloads.make_instance(1000, 20, 100, 10, "1R20", "clustered", seed=1)
    ops, off = workloads.precedence_candidates(1000, 20, 1027, seed=5)
    both(vrp, w, ops, off, sample=[0, 1, 511, 1000, 1026])
