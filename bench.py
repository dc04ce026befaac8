#!/usr/bin/env python3
"""Benchmark of the VRP-RPD hot path on GB300.

Workload (one rank): the n = 1000 instance family -- m = 20 vehicles, pool
R = 100, capacity Q = 10, 1R20 processing times p = round(U_int[1,20] * mean
depot distance / 10), mixed uniform/clustered integer coordinates -- with a
batch of precedence-consistent candidates (every op gets simulated).  A step
evaluates the whole batch (4.2 GB of candidates, larger than L2, so no flush
is needed between steps).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (the slow baseline the ratio is taken against).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

N_CUST, M_VEH, R_POOL, Q_CAP = 1000, 20, 100, 10
BASE_CANDS = 16384          # generated on the host, tiled on the device
# DRAM bytes (read + write) per candidate of each batched kernel, from one ncu
# capture of 16384 candidates of this workload per kernel; a full launch moves
# the same bytes per candidate (the traffic grows in proportion)
TRAFFIC_PER_EVAL = {"eval_tiles_kernel": 8307, "eval_stream_kernel": 8308}
ALNS_OPS_PER_ENTRY = 8
TRAFFIC_SOURCE = "ncu dram__bytes_read+write of a 16384-candidate launch, scaled by candidates per launch"
TILE = 32                   # batch = BASE_CANDS * TILE = 524288 candidates
METRIC = "makespan evals/s and ALNS iters/s at n=1000; batched vs plain GPU, equal makespan"
UNIT = "evals/s"
WORKLOAD = ("n=1000 m=20 R=100 Q=10 1R20 mixed uniform/clustered coords; "
            "524288 precedence-consistent candidates per step (4.24 GB, > L2)")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        # the raw samples go to VRPRPD_CLOCKS_DIR when set (else a temporary
        # directory); their summary is part of the bench line
        out_dir = os.environ.get("VRPRPD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, x, device):
    """The largest x over all ranks (x itself on one rank): the job's time is
    its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second of the slowest rank (every rank
    owns its own shard of the same size: weak scaling)."""
    return units_per_rank * world / seconds


def make_inputs(seed):
    w = workloads.make_instance(N_CUST, M_VEH, R_POOL, Q_CAP, "1R20", "mixed", seed=seed)
    ops, off = workloads.precedence_candidates(N_CUST, M_VEH, BASE_CANDS, seed=seed)
    return w, ops, off


def cpu_baseline(w, ops, off, budget_s=12.0):
    """The oracle as it stands, all host cores, on a bounded sample: whole passes
    over the host candidate set until about budget_s of wall time."""
    import oracle
    oi = oracle.OracleInstance.from_workload(w)
    cores = os.cpu_count() or 1
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.evaluate_batch(oi, ops, off, threads=cores)
        done += len(ops)
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} candidates ({done // len(ops)} passes over {len(ops)}) of the same "
                      f"workload, one C thread per core, {dt:.1f} s"}


def summary_of(line):
    """The headline numbers of every leg in one short object, printed last so
    that a reader of only the line's end still sees them all."""
    def g(*keys):
        x = line
        for k in keys:
            if not isinstance(x, dict) or k not in x:
                return None
            x = x[k]
        return round(x, 4) if isinstance(x, float) else x
    return {
        "evals_per_s_n1000": g("value"), "roofline_frac": g("roofline", "frac"),
        "e2e_evals_per_s": g("e2e", "value"), "plain_gpu_evals_per_s": g("plain_gpu", "value"),
        "ops16_evals_per_s": g("ops16", "value"), "ops16_e2e_evals_per_s": g("ops16", "e2e", "value"),
        "alns_n1000_iters_per_s": g("alns_n1000", "value"), "alns_n1000_iterations": g("alns_n1000", "iterations"),
        "alns_n1000_alu_frac": g("alns_n1000", "roofline", "frac"),
        "alns_n1000_pruned_frac": g("alns_n1000", "pruned_frac"),
        "alns_n1000_x32_iters_per_s": g("alns_n1000_x32", "value"),
        "alns_n100_iters_per_s": g("alns_n100", "value"), "alns_n100_iterations": g("alns_n100", "iterations"),
        "brkga_n200_gens_per_s": g("brkga_n200", "value"), "brkga_n200_generations": g("brkga_n200", "generations"),
        "brkga_n200_hints_gens_per_s": g("brkga_n200_hints", "value"),
        "multi_evals_per_s": g("batched_multi", "value"),
        "serving_req_per_s": g("serving", "value"), "serving_p50_ms": g("serving", "p50_ms"),
        "serving_p99_ms": g("serving", "p99_ms"),
        "serving_c5_completed": g("serving_c5", "completed"), "serving_c5_p50_ms": g("serving_c5", "p50_ms"),
        "serving_c5_p99_ms": g("serving_c5", "p99_ms"),
        "cpu_oracle_evals_per_s": g("cpu_baseline", "value")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, ops, off = make_inputs(seed=0)
    samples = []
    for _ in range(args.warmup):
        cpu_baseline(w, ops, off, budget_s=2.0)
    t_all = time.perf_counter()
    for _ in range(args.steps):
        samples.append(cpu_baseline(w, ops, off, budget_s=max(2.0, 60.0 / max(args.steps, 1))))
    total = time.perf_counter() - t_all
    value = statistics.median(s["value"] for s in samples)
    cb = dict(samples[-1])
    cb["value"] = value
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "sampled subset, CPU"},
        "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                    "d2h_bytes_per_step": 0}}), flush=True)


def run_profile(args):
    """warmup + steps launches of the batched evaluator on the 16384-candidate
    base set (132 MB, larger than L2), default shape; prints per-launch time."""
    import torch
    import paper_2602_23685_gb300 as vrp
    w, ops_h, off_h = make_inputs(seed=0)
    inst = vrp.Instance.from_workload(w)
    if args.profile_walk == "streamed":
        # the shape the autotuner picks for the full batch: two-warp groups of the streamed walk
        vrp.set_eval_config(inst, "coords", 24, walk="streamed", group_warps=2)
    ops = torch.from_numpy(ops_h).cuda()
    off = torch.from_numpy(off_h).cuda()
    for _ in range(args.warmup):
        vrp.evaluate(inst, ops, off)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        z, st = vrp.evaluate(inst, ops, off)
    e1.record()
    vrp.sync(inst)
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"profile_case": "n=1000 m=20, 16384 candidates", "ms_per_launch": ms,
                      "evals_per_s": len(ops_h) / (ms / 1000), "config": vrp.get_eval_config(inst)}))


def run_searches(vrp, args):
    """ALNS iterations/s (n=1000 and the n=100 configuration) and BRKGA
    generations/s (n=200 clustered, pop 1024), each timed on the device."""
    out = {}
    w5 = workloads.make_instance(N_CUST, M_VEH, R_POOL, Q_CAP, "1R20", "mixed", seed=0)
    i5 = vrp.Instance.from_workload(w5)
    vrp.alns_run(i5, vrp.alns_params(2), seed=1)                       # warm-up
    r = vrp.alns_run(i5, vrp.alns_params(args.alns_iters), seed=0)
    st = r["stats"]
    out["alns_n1000"] = {
        "value": args.alns_iters / (st.device_ms / 1000.0), "unit": "ALNS iters/s",
        "config": "n=1000 m=20 R=100 Q=10 1R20, q in [25,50] (Section 4.2.2), greedy+regret-2 over the "
                  "full insertion-delta matrix", "iterations": args.alns_iters,
        "matrix_entries_per_s": st.matrix_entries / (st.device_ms / 1000.0),
        "scored_entries_per_s": (st.matrix_entries - st.pruned_entries) / (st.device_ms / 1000.0),
        "pruned_frac": st.pruned_entries / max(st.matrix_entries, 1),
        "fallback_entries": st.fallback_entries, "team_blocks": st.team_blocks,
        "z_init": st.z_init, "z_best": st.z_best, "device_ms": st.device_ms,
        "phase_ms": dict(zip(["begin", "prep", "gaps", "matrix", "select", "end"], list(st.phase_ms))),
        "incremental_steps": st.incremental_steps, "full_steps": st.full_steps}
    # ALNS moves almost no DRAM bytes: its roofline is integer issue.  Eight
    # integer ops per scored matrix entry (the max-plus formula: three adds and
    # three maxima; the travel add; the compare into the running minimum)
    # against 152 SMs x 128 int32 lanes x 2070 MHz; entries a tile's bound
    # settles without scoring them do no such work and are not counted
    eps = (st.matrix_entries - st.pruned_entries) / (st.device_ms / 1000.0)
    alu_peak = 152 * 128 * 2.07e9 / 1e12
    out["alns_n1000"]["roofline"] = {
        "bound": "alu", "achieved": eps * ALNS_OPS_PER_ENTRY / 1e12, "peak": alu_peak, "unit": "Tops/s",
        "frac": eps * ALNS_OPS_PER_ENTRY / 1e12 / alu_peak, "ops_per_entry": ALNS_OPS_PER_ENTRY,
        "peak_source": "152 SMs x 128 int32 lanes x 2070 MHz (nominal)"}
    # the paper's multi-instance configuration: 32 replicas share the GPU
    # (Section 4.2.1), each a team of 1/32 of the resident CTAs
    rr = vrp.alns_run(i5, vrp.alns_params(args.replica_iters, replicas=32, sync_every=5), seed=0)
    sr = rr["stats"]
    out["alns_n1000_x32"] = {
        "value": 32 * args.replica_iters / (sr.device_ms / 1000.0), "unit": "ALNS iters/s (all replicas)",
        "config": "as alns_n1000 with 32 replicas (multi-instance, Section 4.2.1), best-of-all import every "
                  "5 iterations", "iterations_per_replica": args.replica_iters, "team_blocks": sr.team_blocks,
        "imports": sr.imports, "z_best": sr.z_best, "device_ms": sr.device_ms}
    w2 = workloads.make_instance(100, 4, 10, 5, "2x", "uniform", seed=0)
    i2 = vrp.Instance.from_workload(w2)
    vrp.alns_run(i2, vrp.alns_params(20, 10, 10), seed=1)             # warm-up
    r2 = vrp.alns_run(i2, vrp.alns_params(args.alns100_iters, 10, 10), seed=0)
    st2 = r2["stats"]
    out["alns_n100"] = {
        "value": args.alns100_iters / (st2.device_ms / 1000.0), "unit": "ALNS iters/s",
        "config": "n=100 m=4 R=10 Q=5 2x, q=10; periodic local search (Section 4.2.6) included: pickup "
                  "repositioning every 200 and cross-agent relocation every 500 iterations",
        "iterations": args.alns100_iters,
        "matrix_entries_per_s": st2.matrix_entries / (st2.device_ms / 1000.0),
        "team_blocks": st2.team_blocks, "z_init": st2.z_init, "z_best": st2.z_best,
        "ls_moves": st2.ls_moves, "ls_ms": st2.ls_ms}
    w3 = workloads.make_instance(200, 6, 20, 6, "5x", "clustered", seed=0)
    i3 = vrp.Instance.from_workload(w3)
    a3 = vrp.alns_run(i3, vrp.alns_params(50), seed=0)
    warm = (a3["best_ops"], a3["best_off"])
    vrp.brkga_run(i3, vrp.brkga_params(1024, 2), seed=1, warm=warm)   # warm-up
    t = time.perf_counter()
    b = vrp.brkga_run(i3, vrp.brkga_params(1024, args.brkga_gens), seed=0, warm=warm)
    dt = time.perf_counter() - t
    out["brkga_n200"] = {
        "value": args.brkga_gens / dt, "unit": "BRKGA generations/s",
        "decodes_per_s": args.brkga_gens * 1024 / dt,
        "config": "n=200 clustered m=6 R=20 Q=6 5x, pop 1024, elite 0.2 mutant 0.1 rho 0.7, warm start "
                  "from 50 ALNS iterations", "generations": args.brkga_gens,
        "alns_z": a3["z_best"], "brkga_best": b["best_fitness"]}
    # the paper's 4n chromosome: priorities plus per-op assignment hints (Section 4.4.1)
    hp = vrp.brkga_params(1024, args.brkga_gens, layout=vrp.LAYOUT_HINTS)
    vrp.brkga_run(i3, vrp.brkga_params(1024, 2, layout=vrp.LAYOUT_HINTS), seed=1, warm=warm)   # warm-up
    t = time.perf_counter()
    bh = vrp.brkga_run(i3, hp, seed=0, warm=warm)
    dt = time.perf_counter() - t
    out["brkga_n200_hints"] = {
        "value": args.brkga_gens / dt, "unit": "BRKGA generations/s",
        "decodes_per_s": args.brkga_gens * 1024 / dt,
        "config": "as brkga_n200 with the 4n chromosome (op priorities + assignment hints)",
        "generations": args.brkga_gens, "brkga_best": bh["best_fitness"]}
    return out


def run_multi(vrp, args):
    """256 instances, n log-uniform in [17, 500], m = ceil(n/25), R = ceil(n/10),
    Q = 8, 1R10; 4096 candidates each (512 generated per instance, tiled 8x on
    the device) in one persistent launch replayed as a CUDA graph, against the
    plain form launched once per instance."""
    import torch
    ws = workloads.uneven_instances(256, 17, 500, 8, "1R10", seed=4)
    items = []
    total = 0
    for i, w in enumerate(ws):
        o, f = workloads.precedence_candidates(w.n, w.m, 512, seed=i)
        ops = torch.from_numpy(o).cuda().repeat(8, 1).contiguous()
        off = torch.from_numpy(f).cuda().repeat(8, 1).contiguous()
        items.append((vrp.Instance.from_workload(w), ops, off))
        total += ops.shape[0]
    mb = vrp.MultiBatch(items)
    cfg = mb.autotune()
    stream = torch.cuda.current_stream()
    for _ in range(3):
        mb.evaluate()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(5, args.steps // 5)
    e0.record(stream)
    for _ in range(reps):
        mb.evaluate()
    e1.record(stream)
    torch.cuda.synchronize()
    multi_ms = e0.elapsed_time(e1) / reps
    zs = [z.clone() for z in mb.z]
    outs = []
    for inst, ops, off in items:
        outs.append(vrp.evaluate_plain(inst, ops, off))
    torch.cuda.synchronize()
    e0.record(stream)
    for (inst, ops, off), (zp, sp) in zip(items, outs):
        vrp.evaluate_plain(inst, ops, off, zp, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    equal = all(torch.equal(a, b[0]) for a, b in zip(zs, outs))
    mean_bytes = sum(4 * (2 * w.n + w.m + 1) + 8 for w in ws) / len(ws)
    return {"batched_multi": {
        "value": total / (multi_ms / 1000.0), "unit": "evals/s",
        "config": "256 instances, n log-uniform [17,500], m=ceil(n/25), R=ceil(n/10), Q=8, 1R10; 4096 "
                  "candidates each, one persistent launch replayed as a CUDA graph",
        "candidates_per_launch": total, "ms_per_launch": multi_ms, "eval_config": cfg,
        "achieved_gbs": total * mean_bytes / (multi_ms / 1000.0) / 1e9,
        "plain_per_instance_evals_per_s": total / (plain_ms / 1000.0),
        "speedup_vs_plain": plain_ms / multi_ms, "equal_makespan": equal}}


def run_sweep(vrp, args):
    """Batched evaluation across the configurations' instance shapes (17 to 501
    nodes; base, 2x, 5x and 1R10 processing times): per shape 4096
    precedence-consistent candidates tiled on the device to more than L2, the
    autotuned batched launch timed with CUDA events against the plain form on
    the same batch (equal results asserted), and the HBM fraction of the
    candidate bytes."""
    import torch
    shapes = [(16, 2, 4, 4, "base", "uniform"), (100, 4, 10, 5, "2x", "uniform"),
              (200, 6, 20, 6, "5x", "clustered"), (500, 20, 50, 8, "1R10", "uniform")]
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    stream = torch.cuda.current_stream()
    out = []
    for (n, m, R, Q, variant, layout) in shapes:
        w = workloads.make_instance(n, m, R, Q, variant, layout, seed=7)
        o, f = workloads.precedence_candidates(n, m, 4096, seed=7)
        bpc = 4 * (2 * n + m + 1) + 8
        tiles = -(-(512 << 20) // (4096 * bpc))            # more than L2 per launch
        ops = torch.from_numpy(o).cuda().repeat(tiles, 1).contiguous()
        off = torch.from_numpy(f).cuda().repeat(tiles, 1).contiguous()
        B = ops.shape[0]
        inst = vrp.Instance.from_workload(w)
        # the tuning slice holds four tiles per warp of a full GPU (32 warps per SM)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        tune = min(B, sms * 32 * 4 * max(1, 32 // m))
        cfg = vrp.autotune(inst, ops[:tune], off[:tune])
        z = torch.empty(B, dtype=torch.int32, device="cuda")
        st = torch.empty(B, dtype=torch.int32, device="cuda")
        for _ in range(3):
            vrp.evaluate(inst, ops, off, z, st)
        vrp.sync(inst)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record(stream)
        for _ in range(reps):
            vrp.evaluate(inst, ops, off, z, st)
        e1.record(stream)
        vrp.sync(inst)
        ms = e0.elapsed_time(e1) / reps
        zp, sp = vrp.evaluate_plain(inst, ops, off)
        torch.cuda.synchronize()
        e0.record(stream)
        vrp.evaluate_plain(inst, ops, off, zp, sp)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
        gbs = B * bpc / (ms / 1000.0) / 1e9
        out.append({"workload": f"n={n} m={m} R={R} Q={Q} {variant} {layout}", "batch": B,
                    "value": B / (ms / 1000.0), "unit": UNIT, "achieved_gbs": gbs, "frac": gbs / peak,
                    "plain_evals_per_s": B / (plain_ms / 1000.0), "speedup_vs_plain": plain_ms / ms,
                    "equal_makespan": bool(torch.equal(zp, z)) and bool(torch.equal(sp, st)),
                    "eval_config": cfg})
        del ops, off, z, st, zp, sp, inst
    return {"eval_sweep": {"peak_gbs": peak, "peak_source": "measured" if pk else "fallback",
                           "shapes": out}}


def run_serving(vrp, args, alns_over=None, n_max=400, alns_iters=50, brkga_gens=20):
    """Continuous batching: a Poisson stream of solve requests (n uniform in
    [50, n_max], m = min(20, ceil(n/25)), R = ceil(n/10), Q = 10, 1R20, mixed coords),
    each running alns_iters ALNS iterations then brkga_gens BRKGA generations
    of 256, admitted by a device-memory budget onto 4 concurrent slots.
    Capacity is measured first with all requests queued at once; the stream
    then arrives at 0.8 of that rate and p50/p99 submit-to-finish latency is
    reported."""
    import numpy as np
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(args.serve_requests):
        n = int(rng.integers(50, n_max + 1))
        reqs.append(workloads.make_instance(n, min(20, -(-n // 25)), -(-n // 10), 10, "1R20", "mixed", seed=100 + i))
    budget = 16 << 30

    def run(rate):
        srv = vrp.Server(budget, max_active=4)
        t0 = time.perf_counter()
        ids = []
        for i, w in enumerate(reqs):
            if rate is not None and i:
                time.sleep(float(rng.exponential(1.0 / rate)))
            # the paper's three-phase start, constructor alone (its refinement
            # rounds cost more than 50 iterations at this scale)
            ids.append(srv.submit(w, alns_iterations=alns_iters, brkga_pop=256, brkga_generations=brkga_gens,
                                  seed=i, **(alns_over or {"init_mode": 1, "init_refine_rounds": 0})))
        res = [srv.wait(r) for r in ids]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return res, wall, st

    _, wall0, _ = run(None)
    capacity = len(reqs) / wall0
    res, wall, st = run(0.8 * capacity)
    ok = all(r["status"] == 0 for r in res)
    return {"serving": {
        "value": len(reqs) / wall, "unit": "requests/s", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
        "capacity_requests_per_s": capacity, "arrival_rate": 0.8 * capacity, "requests": len(reqs),
        "peak_active": st["peak_active"], "peak_bytes": st["peak_bytes"], "all_ok": ok,
        "config": f"Poisson arrivals at 0.8x measured capacity; n ~ U[50,{n_max}], m=min(20,ceil(n/25)), "
                  f"R=ceil(n/10), Q=10, 1R20; three-phase start (constructor alone), {alns_iters} ALNS iterations "
                  f"+ {brkga_gens} BRKGA generations of 256 per request; 4 slots, 16 GiB"}}


def run_serving_c5(vrp, args):
    """The full-size serving mix: a Poisson stream of solve requests with n
    uniform in [50, 1000], m = min(20, ceil(n/25)), R = ceil(n/10), Q = 10,
    1R20, mixed coordinates, each running 2000 ALNS iterations then 200 BRKGA
    generations of 1024, admitted by a 32 GiB device-memory budget onto 4
    slots.  The 500-request stream takes far longer than a bench run, so it
    runs in bounded windows: first the capacity (the stream's first requests
    all queued at once for cal_s seconds), then arrivals at 0.8x that rate for
    window_s seconds; requests still waiting for admission at a window's end
    are withdrawn, and those already running finish.  Latencies (submit to
    finish) are over the requests that ran, so the longest requests are
    under-represented when a window cuts the stream."""
    import numpy as np
    rng = np.random.default_rng(11)
    n_req = 500
    ns = rng.integers(50, 1001, size=n_req)
    reqs = [workloads.make_instance(int(n), min(20, -(-int(n) // 25)), -(-int(n) // 10), 10, "1R20", "mixed",
                                    seed=1000 + i) for i, n in enumerate(ns)]
    budget = 32 << 30

    def submit(srv, i):
        return srv.submit(reqs[i], alns_iterations=2000, brkga_pop=1024, brkga_generations=200, seed=i)

    # capacity: everything queued, completions counted over the window
    srv = vrp.Server(budget, max_active=4)
    t0 = time.perf_counter()
    ids = [submit(srv, i) for i in range(min(n_req, 24))]
    while time.perf_counter() - t0 < args.serve_c5_cal and srv.stats()["completed"] < len(ids):
        time.sleep(0.25)
    done_cal = srv.stats()["completed"]
    cal_s = time.perf_counter() - t0
    srv.cancel_pending()
    srv.close()
    capacity = max(done_cal, 1) / cal_s
    rate = 0.8 * capacity
    # the stream at 0.8x capacity, from where the calibration stopped
    srv = vrp.Server(budget, max_active=4)
    t0 = time.perf_counter()
    next_t, i, ids, idx = 0.0, len(ids), [], []
    while i < n_req:
        now = time.perf_counter() - t0
        if now >= args.serve_c5_window:
            break
        if now >= next_t:
            ids.append(submit(srv, i))
            idx.append(i)
            i += 1
            next_t += float(rng.exponential(1.0 / rate))
        else:
            time.sleep(min(0.05, next_t - now))
    withdrawn = srv.cancel_pending()
    res = [srv.wait(r) for r in ids]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    ran_n = [reqs[k].n for k, r in zip(idx, res) if r["status"] == 0]
    return {"serving_c5": {
        "unit": "requests/s", "value": len(ran_n) / wall, "submitted": len(ids), "completed": st["completed"],
        "withdrawn": withdrawn, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
        "capacity_requests_per_s": capacity, "arrival_rate": rate, "window_s": args.serve_c5_window,
        "wall_s": wall, "calibration_s": cal_s, "calibration_completed": done_cal,
        "peak_active": st["peak_active"], "peak_bytes": st["peak_bytes"],
        "mean_n_completed": float(np.mean(ran_n)) if ran_n else None,
        "config": "Poisson arrivals at 0.8x measured capacity; n ~ U[50,1000], m=min(20,ceil(n/25)), "
                  "R=ceil(n/10), Q=10, 1R20, mixed coords; 2000 ALNS iterations + 200 BRKGA generations of "
                  "1024 per request; 4 slots, 32 GiB; bounded window (requests not admitted by its end "
                  "withdrawn)"}}


def run_profile_alns(args):
    """One warm-up ALNS launch and one measured one: n=200 clustered, m=6,
    R=20, Q=6, 5x, 10 iterations; or (--profile-alns-n1000) the n=1000
    workload of the ALNS leg, 2 iterations.  q follows Section 4.2.2."""
    import paper_2602_23685_gb300 as vrp
    if args.profile_alns_n1000:
        w = workloads.make_instance(N_CUST, M_VEH, R_POOL, Q_CAP, "1R20", "mixed", seed=0)
        iters, name = 2, "ALNS n=1000 m=20, 2 iterations"
    else:
        w = workloads.make_instance(200, 6, 20, 6, "5x", "clustered", seed=0)
        iters, name = 10, "ALNS n=200 m=6, 10 iterations"
    inst = vrp.Instance.from_workload(w)
    vrp.alns_run(inst, vrp.alns_params(iters), seed=1)
    r = vrp.alns_run(inst, vrp.alns_params(iters), seed=0)
    st = r["stats"]
    print(json.dumps({"profile_case": name, "device_ms": st.device_ms,
                      "phase_ms": list(st.phase_ms), "incremental_steps": st.incremental_steps,
                      "full_steps": st.full_steps,
                      "iters_per_s": iters / (st.device_ms / 1000), "team_blocks": st.team_blocks,
                      "matrix_entries": st.matrix_entries, "fallback_entries": st.fallback_entries,
                      "pruned_entries": st.pruned_entries, "tiles": st.tiles, "tiles_pruned": st.tiles_pruned}))


def run_profile_brkga(args):
    """The BRKGA leg's instance and warm start (n=200 clustered, 50 ALNS
    iterations), then BRKGA with pop 1024 for 2 generations: two decode
    launches after the initial one."""
    import paper_2602_23685_gb300 as vrp
    w = workloads.make_instance(200, 6, 20, 6, "5x", "clustered", seed=0)
    inst = vrp.Instance.from_workload(w)
    a = vrp.alns_run(inst, vrp.alns_params(50), seed=0)
    warm = (a["best_ops"], a["best_off"])
    t = time.perf_counter()
    b = vrp.brkga_run(inst, vrp.brkga_params(1024, 3), seed=0, warm=warm)
    dt = time.perf_counter() - t
    print(json.dumps({"profile_case": "BRKGA n=200 m=6, pop 1024, 3 generations", "seconds": dt,
                      "best_fitness": b["best_fitness"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-search", action="store_true", help="skip the ALNS / BRKGA legs")
    ap.add_argument("--alns-iters", type=int, default=200, help="ALNS iterations at n=1000")
    ap.add_argument("--alns100-iters", type=int, default=5000, help="ALNS iterations at n=100")
    ap.add_argument("--replica-iters", type=int, default=20, help="iterations per replica, 32 replicas at n=1000")
    ap.add_argument("--brkga-gens", type=int, default=1000)
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-c5-window", type=float, default=90.0,
                    help="seconds of Poisson arrivals in the full-size serving leg (0 = skip the leg)")
    ap.add_argument("--serve-c5-cal", type=float, default=45.0,
                    help="seconds of the full-size serving leg's capacity measurement")
    ap.add_argument("--profile-alns", action="store_true",
                    help="small ALNS case for ncu: n=200, 10 iterations per launch, one warm-up launch")
    ap.add_argument("--profile-brkga", action="store_true",
                    help="small BRKGA case for ncu: n=200, pop 1024, 3 generations from the ALNS warm start")
    ap.add_argument("--profile-alns-n1000", action="store_true",
                    help="small ALNS case for ncu on the n=1000 workload: 2 iterations per launch")
    ap.add_argument("--profile", action="store_true",
                    help="small case for ncu: 16384 candidates (132 MB), no tuning")
    ap.add_argument("--profile-walk", default="staged", choices=["staged", "streamed"],
                    help="--profile: the default staged shape, or the streamed two-warp-group shape")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    if args.profile_alns or args.profile_alns_n1000:
        return run_profile_alns(args)
    if args.profile_brkga:
        return run_profile_brkga(args)

    import torch
    import paper_2602_23685_gb300 as vrp

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w, ops_h, off_h = make_inputs(seed=rank)
    inst = vrp.Instance.from_workload(w)
    base_ops = torch.from_numpy(ops_h).cuda()
    base_off = torch.from_numpy(off_h).cuda()
    ops = base_ops.repeat(TILE, 1).contiguous()
    off = base_off.repeat(TILE, 1).contiguous()
    B = ops.shape[0]
    z = torch.empty(B, dtype=torch.int32, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    tuned = vrp.autotune(inst, ops[: BASE_CANDS * 4], off[: BASE_CANDS * 4])
    for _ in range(args.warmup):
        vrp.evaluate(inst, ops, off, z, st)
    vrp.sync(inst)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            starts[i].record(stream)
            vrp.evaluate(inst, ops, off, z, st)
            ends[i].record(stream)
        t1.record(stream)
        barrier()
    vrp.sync(inst)
    total_ms = t0.elapsed_time(t1)
    kernel_ms = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    value = whole_job_rate(B * args.steps, world, total_ms / 1000.0)

    # correctness of the timed output: first tile against the plain GPU form, and
    # every tiled copy identical to the first
    zc, sc = z.view(TILE, BASE_CANDS), st.view(TILE, BASE_CANDS)
    assert bool((zc == zc[0]).all()) and bool((sc == sc[0]).all())

    # plain per-instance GPU form on the same batch, fewer steps
    zp = torch.empty_like(z)
    sp = torch.empty_like(st)
    vrp.evaluate_plain(inst, ops, off, zp, sp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_steps = 3
    e0.record(stream)
    for _ in range(plain_steps):
        vrp.evaluate_plain(inst, ops, off, zp, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_value = B * plain_steps / (e0.elapsed_time(e1) / 1000.0)
    equal = bool(torch.equal(zp, z)) and bool(torch.equal(sp, st))

    # end to end: pinned host candidates -> device -> evaluate -> host results
    e2e_steps = max(3, min(10, args.steps))
    ops_pin = ops.cpu().pin_memory()
    off_pin = off.cpu().pin_memory()
    z_h = torch.empty(B, dtype=torch.int32).pin_memory()
    st_h = torch.empty(B, dtype=torch.int32).pin_memory()
    vrp.evaluate_host(inst, ops_pin, off_pin, z_h, st_h)
    barrier()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        vrp.evaluate_host(inst, ops_pin, off_pin, z_h, st_h)
    barrier()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t, "cuda")
    e2e_value = whole_job_rate(B * e2e_steps, world, e2e_s)
    assert torch.equal(z_h, z.cpu())

    # the host link's own rate: a pinned host -> device copy of the step's
    # candidate bytes, the ceiling of any end-to-end path that moves them
    scratch = torch.empty_like(ops)
    link_ms = []
    for _ in range(3):
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        scratch.copy_(ops_pin, non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize()
        link_ms.append(l0.elapsed_time(l1))
    del scratch
    link_gbs = ops.numel() * 4 / (min(link_ms[1:]) / 1000.0) / 1e9
    e2e_bytes = int(ops.numel() * 4 + off.numel() * 4)
    e2e_gbs = e2e_bytes * e2e_steps / e2e_s / 1e9          # per GPU, like its link

    # the 16-bit form: the same candidates as 16-bit codes and offsets (half
    # the bytes), on the device and end to end from pinned host memory
    ops16, off16 = ops.to(torch.int16), off.to(torch.int16)
    z16, st16 = torch.empty_like(z), torch.empty_like(st)
    vrp.evaluate(inst, ops16, off16, z16, st16)
    vrp.sync(inst)
    assert torch.equal(z16, z) and torch.equal(st16, st)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(e2e_steps):
        vrp.evaluate(inst, ops16, off16, z16, st16)
    s1.record(stream)
    vrp.sync(inst)
    w16_value = whole_job_rate(B * e2e_steps, world, max_over_ranks(dist, s0.elapsed_time(s1), "cuda") / 1000.0)
    ops16_pin, off16_pin = ops16.cpu().pin_memory(), off16.cpu().pin_memory()
    del ops16, off16
    vrp.evaluate_host(inst, ops16_pin, off16_pin, z_h, st_h)
    barrier()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        vrp.evaluate_host(inst, ops16_pin, off16_pin, z_h, st_h)
    barrier()
    e2e16_s = max_over_ranks(dist, time.perf_counter() - t, "cuda")
    assert torch.equal(z_h, z.cpu())
    e2e16_bytes = int(ops16_pin.numel() * 2 + off16_pin.numel() * 2)
    ops16_leg = {"ops16": {
        "value": w16_value, "unit": UNIT,
        "config": "the same batch as 16-bit op codes and offsets (vrprpd_evaluate16), results equal",
        "e2e": {"value": whole_job_rate(B * e2e_steps, world, e2e16_s), "unit": UNIT,
                "h2d_bytes_per_step": e2e16_bytes, "d2h_bytes_per_step": int(B * 8),
                "link_frac": e2e16_bytes * e2e_steps / e2e16_s / 1e9 / link_gbs}}}
    del ops16_pin, off16_pin

    # Section 5.2 coordination counts over the first quarter of the batch:
    # same candidate bytes read, a lock-step walk per candidate like the
    # evaluator's; every tiled copy must give the first copy's counts
    Bc = B // 4
    cr, il = vrp.coordination(inst, ops[:Bc], off[:Bc])
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    co_steps = 3
    c0.record(stream)
    for _ in range(co_steps):
        cr, il = vrp.coordination(inst, ops[:Bc], off[:Bc])
    c1.record(stream)
    torch.cuda.synchronize()
    co_ms = c0.elapsed_time(c1) / co_steps
    crv, ilv = cr.view(-1, BASE_CANDS), il.view(-1, BASE_CANDS)
    coordination = {"coordination_counts": {
        "value": Bc / (co_ms / 1000.0), "unit": "candidates/s", "candidates": Bc, "ms": co_ms,
        "kernel": "coordination_kernel", "tiles_agree": bool((crv == crv[0]).all()) and bool((ilv == ilv[0]).all()),
        "mean_cross_pct": float(cr.double().mean()) * 100.0 / N_CUST,
        "mean_interleaved_pct": float(il.double().mean()) * 100.0 / N_CUST}}

    searches = {} if args.no_search else run_searches(vrp, args)
    searches.update(coordination)
    if not args.no_search:
        searches.update(run_sweep(vrp, args))
        searches.update(run_multi(vrp, args))
        searches.update(run_serving(vrp, args))
        if args.serve_c5_window > 0:
            searches.update(run_serving_c5(vrp, args))

    pk = peaks()
    bytes_per_eval = 4 * (2 * N_CUST + M_VEH + 1) + 8
    achieved = B * bytes_per_eval / (kernel_ms / 1000.0) / 1e9
    peak = pk["hbm_gbs"] if pk else 6800.0
    kernel = "eval_stream_kernel" if tuned.get("walk") == "streamed" else "eval_tiles_kernel"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured" if pk else "fallback",
                "bytes_per_unit": bytes_per_eval, "units_per_launch": B,
                "traffic": TRAFFIC_PER_EVAL[kernel] * B, "traffic_source": TRAFFIC_SOURCE,
                "kernel": kernel, "kernel_ms": kernel_ms}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": B, "l2": "inputs larger than L2 (no flush)",
                       "eval_config": tuned},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes,
                    "d2h_bytes_per_step": int(B * 8), "link_gbs": link_gbs, "link_frac": e2e_gbs / link_gbs,
                    "link_source": "pinned host -> device copy of the step's ops, CUDA events"},
            "gpu_launches": args.steps,
            "roofline": roofline,
            "clocks": clk.summary(),
            "plain_gpu": {"value": plain_value, "unit": UNIT, "equal_makespan": equal,
                          "speedup_batched_vs_plain": value / world / plain_value},
        }
        line.update(ops16_leg)
        line.update(searches)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, ops_h, off_h)
        line["summary"] = summary_of(line)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
