"""GPU parity of candidate evaluation against the CPU oracle: bit-exact makespan
and status for every candidate, every distance mode, the plain form and the
host-buffer path; ragged tiles, odd n (unaligned TMA), m = 1 and m = 32,
malformed and cyclic candidates, and the full-size n = 1000 workload."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

MODES = ["smem32", "smem16", "global16", "global32", "coords"]


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# each distance mode runs with the staged walk and with the streamed walk in
# groups of one and of two warps
WALKS = [("staged", 1), ("streamed", 1), ("streamed", 2)]


def run_modes(vrp, inst, ops, off, modes=MODES):
    results = {}
    for mode in modes:
        for walk, gw in WALKS:
            try:
                vrp.set_eval_config(inst, mode, 8, walk=walk, group_warps=gw)
            except vrp.VrpError:
                continue
            z, st = vrp.evaluate(inst, dev(ops), dev(off))
            vrp.sync(inst)
            results[f"{mode}/{walk}{gw}"] = (z.cpu().numpy(), st.cpu().numpy().astype(np.uint32))
    vrp.set_eval_config(inst, "auto")
    return results


def check_against_oracle(vrp, w, ops, off, modes=MODES, load_full=False, threads=8):
    inst = vrp.Instance.from_workload(w, load_full=load_full)
    oi = oracle.OracleInstance.from_workload(w, load_full=load_full)
    assert np.array_equal(inst.dist(), oracle.euc2d(w.coords))
    zo, so = oracle.evaluate_batch(oi, ops, off, threads=threads)
    res = run_modes(vrp, inst, ops, off, modes)
    assert res, "no distance mode ran"
    for mode, (z, st) in res.items():
        bad = np.nonzero((z != zo) | (st != so))[0]
        assert bad.size == 0, (mode, bad[:5], z[bad[:5]], zo[bad[:5]], st[bad[:5]], so[bad[:5]])
    zp, sp = vrp.evaluate_plain(inst, dev(ops), dev(off))
    assert np.array_equal(zp.cpu().numpy(), zo) and np.array_equal(sp.cpu().numpy().astype(np.uint32), so)
    return inst, zo, so


def test_n16_random_and_precedence(vrp):
    cfg = workloads.CONFIGS["tiny_n16"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], seed=0)
    ops, off = workloads.random_candidates(w.n, w.m, 4096, seed=0)
    _, zo, so = check_against_oracle(vrp, w, ops, off)
    assert (so & oracle.CYCLE).any()                     # random orders are mostly cyclic
    ops, off = workloads.precedence_candidates(w.n, w.m, 4096, seed=1)
    _, zo, so = check_against_oracle(vrp, w, ops, off)
    assert not (so & oracle.CYCLE).any()


def test_n100_full_batch(vrp):
    cfg = workloads.CONFIGS["alns_n100"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], seed=0)
    ops, off = workloads.precedence_candidates(w.n, w.m, 65536, seed=2)
    check_against_oracle(vrp, w, ops, off, modes=["smem32", "coords"])


@pytest.mark.parametrize("n,m,count", [(1, 1, 5), (1, 2, 7), (7, 3, 333), (33, 32, 65), (51, 1, 40),
                                       (101, 5, 1001), (200, 6, 257)])
def test_shapes_ragged_and_odd(vrp, n, m, count):
    w = workloads.make_instance(n, m, R=max(1, n // 3), Q=3, variant="2x", seed=n)
    o1, f1 = workloads.precedence_candidates(n, m, count, seed=5)
    o2, f2 = workloads.random_candidates(n, m, count, seed=6)
    ops = np.concatenate([o1, o2])
    off = np.concatenate([f1, f2])
    check_against_oracle(vrp, w, ops, off)
    # an offset view into the batch: the op array no longer starts 16-byte aligned
    import torch
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    big = dev(np.concatenate([np.full((1, 2 * n), 2, np.int32), ops]).reshape(-1))
    sub = big[2 * n:].view(-1, 2 * n)
    if n % 2 == 1:
        assert (sub.data_ptr() % 16) != 0
    z, st = vrp.evaluate(inst, sub, dev(off))
    zo, so = oracle.evaluate_batch(oi, ops, off, threads=8)
    assert np.array_equal(z.cpu().numpy(), zo) and np.array_equal(st.cpu().numpy().astype(np.uint32), so)


def test_load_full(vrp):
    w = workloads.make_instance(40, 4, R=40, Q=6, seed=9)
    ops, off = workloads.precedence_candidates(40, 4, 2000, seed=9)
    check_against_oracle(vrp, w, ops, off, load_full=True)


def test_malformed_candidates(vrp):
    n, m = 10, 3
    w = workloads.make_instance(n, m, R=5, Q=3, seed=4)
    ops, off = workloads.precedence_candidates(n, m, 64, seed=4)
    ops = ops.copy()
    off = off.copy()
    ops[0, 3] = ops[0, 4]                  # duplicate op
    ops[1, 0] = 2 * n + 2                  # op code out of range
    ops[2, 5] = 1                          # op code below range
    off[3, 1], off[3, 2] = off[3, 2], off[3, 1] + 0  # possibly decreasing
    off[3, 1] = off[3, 2] + 1
    off[4, 0] = 1                          # off[0] != 0
    off[5, m] = 2 * n - 1                  # off[m] != 2n
    inst, zo, so = check_against_oracle(vrp, w, ops, off)
    assert all(so[i] == oracle.MALFORMED for i in range(6))


def test_duplicate_and_missing_ops(vrp):
    # one op overwritten by a copy of another: a repeated code and a missing
    # one, drops or pickups, on one route or across routes, in acyclic and
    # cyclic candidates; plus two routes that start with the same drop (the
    # duplicate reaches both lanes in the same step)
    n, m = 30, 5
    w = workloads.make_instance(n, m, 12, 4, "2x", seed=9)
    rng = np.random.default_rng(9)
    po, pf = workloads.precedence_candidates(n, m, 1500, seed=9)
    ro, rf = workloads.random_candidates(n, m, 1500, seed=10)
    ops, off = np.concatenate([po, ro]).copy(), np.concatenate([pf, rf])
    for k in range(len(ops)):
        i, j = rng.choice(2 * n, size=2, replace=False)
        ops[k, i] = ops[k, j]
    for k in range(0, 200):
        if off[k, 1] > off[k, 0] and off[k, 2] > off[k, 1]:
            ops[k, off[k, 1]] = ops[k, off[k, 0]]
    inst, zo, so = check_against_oracle(vrp, w, ops, off)
    assert (so == oracle.MALFORMED).all()


def _boundary_chain(n, seed):
    """Depot at the centre of a 2895-wide box and n customers on a chain whose
    consecutive legs have squared lengths on EUC_2D's rounding boundaries:
    s = r^2 - r or r^2 + r (just below r -+ 1/2) and s = r^2 - r + 1 or
    r^2 + r + 1 (just above), for 2 <= r <= 2040.  Every step moves toward the
    centre, so the box (squared diagonal < 2^24) is never left."""
    import math
    rng = np.random.default_rng(seed)
    pts = [(1448, 1448)]
    while len(pts) <= n:
        r = int(rng.integers(2, 2041))
        s = r * r + int(rng.choice([-r, -r + 1, r, r + 1]))
        reps = [(dx, math.isqrt(s - dx * dx)) for dx in range(0, math.isqrt(s) + 1)
                if math.isqrt(s - dx * dx) ** 2 == s - dx * dx]
        reps = [(dx, dy) for dx, dy in reps if dx <= 1447 and dy <= 1447]
        if not reps:
            continue
        dx, dy = reps[int(rng.integers(0, len(reps)))]
        x, y = pts[-1]
        pts.append((x + (dx if x <= 1448 else -dx), y + (dy if y <= 1448 else -dy)))
    coords = np.array(pts, dtype=np.int32)
    leg = np.diff(coords.astype(np.int64), axis=0)
    s = (leg ** 2).sum(axis=1)
    r = np.array([math.isqrt(int(v)) for v in s])
    gap = s - (r * r + r)
    assert ((gap == 0) | (gap == 1)).all() and coords.min() >= 0 and coords.max() <= 2895
    return coords


def test_rounding_boundary_legs(vrp):
    # makespans over chains of legs whose exact EUC_2D rounding is closest to
    # a tie.  m = 32: one long route takes 1469 consecutive chain legs (it
    # sets the makespan, so every one of its legs is in the result), the other
    # 31 routes one customer each; its rotations move the cut.  m = 20: the
    # chain cut into random routes.
    n, m = 1500, 32
    coords = _boundary_chain(n, seed=5)
    p = np.random.default_rng(6).integers(0, 200, size=n).astype(np.int32)
    chain = np.arange(1, n + 1)
    ops1 = []
    for k in range(0, n, 47):
        order = np.roll(chain, -k)
        ops1.append(np.stack([2 * order, 2 * order + 1], axis=1).reshape(-1))
    ops1 = np.array(ops1, dtype=np.int32)
    long = 2 * (n - (m - 1))
    off1 = np.tile(np.concatenate([[0], np.arange(long, 2 * n + 1, 2)]).astype(np.int32), (len(ops1), 1))
    assert off1.shape[1] == m + 1
    inst, zo, so = check_against_oracle(vrp, workloads.Instance(coords, p, m, m, 2), ops1, off1)
    assert (so == 0).all() and (zo > 1000 * n // 2).all()
    m = 20
    cuts = np.sort(np.random.default_rng(7).integers(0, n + 1, size=(64, m - 1)), axis=1)
    off2 = np.concatenate([np.zeros((64, 1), np.int64), 2 * cuts, np.full((64, 1), 2 * n)], axis=1)
    ops2 = np.tile(ops1[0], (64, 1))
    check_against_oracle(vrp, workloads.Instance(coords, p, m, m, 2), ops2, off2.astype(np.int32))


def test_host_path_matches(vrp):
    w = workloads.make_instance(100, 4, 10, 5, "2x", seed=1)
    inst = vrp.Instance.from_workload(w)
    ops, off = workloads.precedence_candidates(100, 4, 3000, seed=8)
    z1, s1 = vrp.evaluate(inst, dev(ops), dev(off))
    z2, s2 = vrp.evaluate_host(inst, ops, off)
    assert np.array_equal(z1.cpu().numpy(), z2) and np.array_equal(s1.cpu().numpy().astype(np.uint32), s2)


def test_pinned_host_path_reads_in_place(vrp):
    # pinned buffers: the kernel reads the ops over the host link, no staging copy
    import torch
    for (n, m, seed) in ((100, 4, 2), (37, 5, 4), (1000, 20, 6)):
        w = workloads.make_instance(n, m, 10, 5, "2x", seed=seed)
        inst = vrp.Instance.from_workload(w)
        oi = oracle.OracleInstance.from_workload(w)
        ops, off = workloads.precedence_candidates(n, m, 700, seed=seed)
        rops, roff = workloads.random_candidates(n, m, 300, seed=seed)
        ops, off = np.concatenate([ops, rops]), np.concatenate([off, roff])
        ops[5, 3] = ops[5, 4]                      # a repeated op
        off[6, m] = 2 * n - 1                      # offsets that end short
        tops = torch.from_numpy(ops).pin_memory()
        toff = torch.from_numpy(off).pin_memory()
        z, st = vrp.evaluate_host(inst, tops, toff)
        zo, so = oracle.evaluate_batch(oi, ops, off, threads=8)
        assert np.array_equal(z, zo) and np.array_equal(st, so)


def _as16(a):
    assert a.min() >= 0 and a.max() < 65536
    return a.astype(np.uint16).view(np.int16)


@pytest.mark.parametrize("n,m,count,seed", [(17, 2, 333, 1), (100, 4, 1000, 2), (37, 1, 70, 3),
                                            (61, 32, 45, 4), (1000, 20, 300, 5)])
def test_sixteen_bit_form(vrp, n, m, count, seed):
    # the same codes and offsets as 16-bit values: device, pageable host and
    # pinned host paths all equal the oracle on the 32-bit values, in every
    # distance mode, malformed candidates included (codes 0, 1, 2n+2 and 65535,
    # a repeated code, offsets past 2n or decreasing)
    import torch
    w = workloads.make_instance(n, m, max(m, 10), 5, "2x", seed=seed)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    po, pf = workloads.precedence_candidates(n, m, count, seed=seed)
    ro, rf = workloads.random_candidates(n, m, count, seed=seed + 50)
    ops, off = np.concatenate([po, ro]).copy(), np.concatenate([pf, rf]).copy()
    ops[0, 0], ops[1, 1], ops[2, 2], ops[3, 2 * n - 1] = 0, 1, 2 * n + 2, 65535
    ops[4, 3] = ops[4, 4]
    off[5, m] = 2 * n + 1
    if m > 1:
        off[6, 1] = off[6, 2] + 1
    zo, so = oracle.evaluate_batch(oi, ops, off, threads=8)
    assert (so[:6] == oracle.MALFORMED).all()
    o16, f16 = _as16(ops), _as16(off)
    res = run_modes(vrp, inst, o16, f16)
    assert res
    for mode, (z, st) in res.items():
        assert np.array_equal(z, zo) and np.array_equal(st, so), mode
    z, st = vrp.evaluate_host(inst, o16, f16)
    assert np.array_equal(z, zo) and np.array_equal(st, so)
    z, st = vrp.evaluate_host(inst, torch.from_numpy(o16).pin_memory(), torch.from_numpy(f16).pin_memory())
    assert np.array_equal(z, zo) and np.array_equal(st, so)


def test_sixteen_bit_form_rejects_mixed_widths(vrp):
    w = workloads.make_instance(20, 2, 4, 4, seed=1)
    inst = vrp.Instance.from_workload(w)
    ops, off = workloads.precedence_candidates(20, 2, 8, seed=1)
    with pytest.raises(TypeError):
        vrp.evaluate(inst, dev(_as16(ops)), dev(off))
    with pytest.raises(TypeError):
        vrp.evaluate_host(inst, ops, _as16(off))
    with pytest.raises(TypeError):
        vrp.evaluate_plain(inst, dev(_as16(ops)), dev(_as16(off)))


def test_autotune_keeps_results(vrp):
    w = workloads.make_instance(100, 4, 10, 5, "2x", seed=3)
    inst = vrp.Instance.from_workload(w)
    ops, off = workloads.precedence_candidates(100, 4, 8192, seed=3)
    z1, s1 = vrp.evaluate(inst, dev(ops), dev(off))
    cfg = vrp.autotune(inst, dev(ops), dev(off))
    assert cfg["dist_mode"] in MODES
    z2, s2 = vrp.evaluate(inst, dev(ops), dev(off))
    assert np.array_equal(z1.cpu().numpy(), z2.cpu().numpy())
    assert np.array_equal(s1.cpu().numpy(), s2.cpu().numpy())


@pytest.mark.parametrize("seed", [0, 1])
def test_n1000_full_size_sampled(vrp, seed):
    # the headline workload: n = 1000, m = 20, R = 100, Q = 10, 1R20 processing times;
    # a 4096-candidate batch on the device, the oracle checks every 8th candidate
    cfg = workloads.CONFIGS["serving_n1000"]
    w = workloads.make_instance(cfg["n"], cfg["m"], cfg["R"], cfg["Q"], cfg["variant"], cfg["layout"], seed=seed)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    assert np.array_equal(inst.dist(), oracle.euc2d(w.coords))
    ops, off = workloads.precedence_candidates(w.n, w.m, 4096, seed=seed)
    idx = np.arange(0, 4096, 8)
    zo, so = oracle.evaluate_batch(oi, ops[idx], off[idx], threads=8)
    shapes = [("coords", 4, "staged", 1), ("global16", 4, "staged", 1), ("global32", 4, "staged", 1),
              ("coords", 30, "streamed", 2), ("coords", 16, "streamed", 1), ("global16", 8, "streamed", 2),
              ("auto", 0, "staged", 1)]
    for mode, warps, walk, gw in shapes:
        vrp.set_eval_config(inst, mode, warps, walk=walk, group_warps=gw)
        z, st = vrp.evaluate(inst, dev(ops), dev(off))
        vrp.sync(inst)
        assert np.array_equal(z.cpu().numpy()[idx], zo), (mode, walk, gw)
        assert np.array_equal(st.cpu().numpy().astype(np.uint32)[idx], so), (mode, walk, gw)
    # the shape the autotuner picks (the one the benchmark times)
    cfg = vrp.autotune(inst, dev(ops), dev(off))
    z, st = vrp.evaluate(inst, dev(ops), dev(off))
    vrp.sync(inst)
    assert np.array_equal(z.cpu().numpy()[idx], zo), cfg
    assert np.array_equal(st.cpu().numpy().astype(np.uint32)[idx], so), cfg
    vrp.set_eval_config(inst, "auto")


def test_repeated_op_across_warps_same_step(vrp):
    """The streamed walk with two-warp groups at m = 20 packs three candidates
    onto 64 lanes: candidate 1 of a group has routes 0-11 on the first warp
    and routes 12-19 on the second.  Two routes that start with the same drop
    (or the same pickup right after the same drop) on different warps reach
    it in the same step; the exchange on the ready slot must still catch the
    repeat (MALFORMED, as the oracle says)."""
    n, m = 60, 20
    w = workloads.make_instance(n, m, 60, 6, "2x", seed=21)
    ops, off = workloads.precedence_candidates(n, m, 300, seed=21)
    ops, off = ops.copy(), off.copy()
    changed = []
    for k in range(len(ops)):
        if k % 3 != 1:
            continue
        r0, r15 = (0, 15) if k % 2 else (3, 17)
        if off[k, r0 + 1] > off[k, r0] and off[k, r15 + 1] > off[k, r15]:
            ops[k, off[k, r15]] = ops[k, off[k, r0]]
            changed.append(k)
    assert len(changed) > 50
    inst, zo, so = check_against_oracle(vrp, w, ops, off)
    assert (so[changed] == oracle.MALFORMED).all()


def test_streamed_groups_repeatable(vrp):
    """Two-warp groups meet once per step; a warp that leaves the barrier first
    may start the next step before its partner has read this step's progress.
    Many launches of mostly cyclic and acyclic candidates at m = 20 (one
    candidate of each group split across the two warps), in several block
    shapes, must all equal the oracle."""
    n, m = 80, 20
    w = workloads.make_instance(n, m, 80, 6, "2x", seed=31)
    po, pf = workloads.precedence_candidates(n, m, 1500, seed=31)
    ro, rf = workloads.random_candidates(n, m, 1500, seed=32)
    ops, off = np.concatenate([po, ro]), np.concatenate([pf, rf])
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    zo, so = oracle.evaluate_batch(oi, ops, off, threads=8)
    assert (so & oracle.CYCLE).any() and not (so[:1500] & oracle.CYCLE).any()
    do, df = dev(ops), dev(off)
    for warps in (2, 8, 24):
        vrp.set_eval_config(inst, "coords", warps, walk="streamed", group_warps=2)
        for _ in range(8):
            z, st = vrp.evaluate(inst, do, df)
            vrp.sync(inst)
            assert np.array_equal(z.cpu().numpy(), zo) and np.array_equal(st.cpu().numpy().astype(np.uint32), so), warps
    vrp.set_eval_config(inst, "auto")
