"""ctypes front end of the VRP-RPD CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package.  Every function here forwards to the plain C oracle in
this directory (see oracle.h for the paper passages each one follows).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["evaluate.c", "exact.c", "search.c"]
_lock = threading.Lock()
_lib = None

CYCLE, VEH_CAP, POOL, MALFORMED = 1, 2, 4, 8
LOAD_FULL = 1


def build(force=False):
    """Compile liboracle.so with gcc (no FMA contraction, so its fp64 search
    arithmetic rounds exactly as written)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Inst(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("R", C.c_int32), ("Q", C.c_int32),
                ("flags", C.c_uint32), ("d", C.POINTER(C.c_int32)), ("p", C.POINTER(C.c_int32))]


class AlnsParams(C.Structure):
    _fields_ = [("T0", C.c_double), ("alpha", C.c_double), ("reheat", C.c_double),
                ("r", C.c_double), ("stagnation", C.c_int32), ("tau", C.c_int32),
                ("sigma1", C.c_int32), ("sigma2", C.c_int32), ("sigma3", C.c_int32),
                ("w_min", C.c_double), ("q_min", C.c_int32), ("q_max", C.c_int32),
                ("iterations", C.c_int32), ("repair_mask", C.c_int32), ("destroy_mask", C.c_int32),
                ("ls_pickup_every", C.c_int32), ("ls_relocate_every", C.c_int32)]


class AlnsStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accepted", C.c_int32), ("improved", C.c_int32),
                ("new_best", C.c_int32), ("reheats", C.c_int32),
                ("rejected_infeasible", C.c_int32), ("z_init", C.c_int32),
                ("z_best", C.c_int32), ("z_current", C.c_int32), ("T_final", C.c_double),
                ("w_destroy", C.c_double * 8), ("w_repair", C.c_double * 4),
                ("ls_moves", C.c_int32), ("ls_new_best", C.c_int32)]


class BrkgaParams(C.Structure):
    _fields_ = [("pop", C.c_int32), ("generations", C.c_int32), ("warm_slots", C.c_int32),
                ("warm_variants", C.c_int32), ("elite_frac", C.c_float),
                ("mutant_frac", C.c_float), ("rho", C.c_float), ("eps", C.c_float),
                ("layout", C.c_int32)]


LAYOUT_VKEYS = 0   # 2n priority keys + m vehicle keys
LAYOUT_HINTS = 1   # 2n priority keys + 2n assignment hints (Section 4.4.1)


def key_length(I, layout):
    return 4 * I.n if layout == LAYOUT_HINTS else 2 * I.n + I.m


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            i32p, u32p, i64p = C.POINTER(C.c_int32), C.POINTER(C.c_uint32), C.POINTER(C.c_int64)
            f32p = C.POINTER(C.c_float)
            L.oracle_euc2d.argtypes = [i32p, C.c_int32, i32p]
            L.oracle_evaluate.argtypes = [C.POINTER(Inst), i32p, i32p, C.c_int, i32p, u32p, i64p]
            L.oracle_evaluate_batch.argtypes = [C.POINTER(Inst), C.c_int32, i32p, i32p, i32p, u32p,
                                                C.c_int32]
            L.oracle_sp_closure.argtypes = [i32p, C.c_int32, i64p]
            L.oracle_coordination.argtypes = [C.POINTER(Inst), i32p, i32p, i32p, i32p]
            L.oracle_coordination.restype = C.c_uint32
            L.oracle_initial_solution_paper.argtypes = [C.POINTER(Inst), i32p, C.c_int32, i32p, i32p]
            L.oracle_alns_run_replicas.argtypes = [C.POINTER(Inst), i32p, i32p, C.POINTER(AlnsParams), C.c_uint64,
                                                   C.c_int32, C.c_int32, i32p, i32p, i32p,
                                                   C.POINTER(AlnsStats), i32p, i32p]
            L.oracle_seed_chromosome.argtypes = [C.POINTER(Inst), C.c_int32, C.c_int32, f32p]
            L.oracle_local_search.argtypes = [C.POINTER(Inst), C.c_int32, C.c_int32, i32p, i32p, i32p]
            L.oracle_bruteforce.argtypes = [C.POINTER(Inst), i32p, i32p]
            L.oracle_bruteforce.restype = C.c_int64
            L.oracle_minmax_vrp.argtypes = [i32p, C.c_int32, C.c_int32]
            L.oracle_minmax_vrp.restype = C.c_int64
            L.oracle_held_karp.argtypes = [i32p, C.c_int32]
            L.oracle_held_karp.restype = C.c_int64
            L.oracle_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
            L.oracle_splitmix64_next.restype = C.c_uint64
            L.oracle_rng.argtypes = [C.c_uint64, C.c_uint64]
            L.oracle_rng.restype = C.c_uint64
            L.oracle_exp.argtypes = [C.c_double]
            L.oracle_exp.restype = C.c_double
            L.oracle_q_range.argtypes = [C.c_int32, i32p, i32p]
            L.oracle_insertion_matrix.argtypes = [C.POINTER(Inst), i32p, i32p, C.c_int32, i32p, i32p,
                                                  u32p]
            L.oracle_initial_solution.argtypes = [C.POINTER(Inst), i32p, i32p, i32p]
            L.oracle_alns_run.argtypes = [C.POINTER(Inst), i32p, i32p, C.POINTER(AlnsParams),
                                          C.c_uint64, i32p, i32p, i32p, i32p, C.POINTER(AlnsStats),
                                          i32p]
            L.oracle_decode.argtypes = [C.POINTER(Inst), f32p, i32p, i32p, i32p, i32p, i64p]
            L.oracle_encode.argtypes = [C.POINTER(Inst), i32p, i32p, f32p]
            L.oracle_destroy.argtypes = [C.POINTER(Inst), C.c_int32, i32p, i32p, C.c_int32, C.c_int32,
                                         C.c_uint64, C.c_uint64, C.c_char_p]
            L.oracle_decode_l.argtypes = [C.POINTER(Inst), f32p, C.c_int32, i32p, i32p, i32p, i32p, i64p]
            L.oracle_encode_l.argtypes = [C.POINTER(Inst), i32p, i32p, C.c_int32, f32p]
            L.oracle_brkga_run.argtypes = [C.POINTER(Inst), C.POINTER(BrkgaParams), i32p, i32p,
                                           C.c_uint64, f32p, i64p, i32p, i32p, i64p]
            L.oracle_repair.argtypes = [C.POINTER(Inst), C.c_int32, i32p, i32p, i32p, C.c_int32, C.c_int32,
                                        i32p, i32p]
            f64p = C.POINTER(C.c_double)
            L.oracle_alns_adapt_script.argtypes = [C.POINTER(AlnsParams), C.c_int32, C.c_int32, i32p, i32p,
                                                   i32p, u32p, f64p, C.POINTER(AlnsStats), i32p]
            _lib = L
    return _lib


def _p(a, ct=C.c_int32):
    return a.ctypes.data_as(C.POINTER(ct))


def euc2d(coords):
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    N = coords.shape[0]
    d = np.empty((N, N), dtype=np.int32)
    lib().oracle_euc2d(_p(coords), N, _p(d))
    return d


class OracleInstance:
    """Holds d, p and sizes for the C oracle; keeps the arrays alive."""

    def __init__(self, d, p, m, R, Q, load_full=False):
        self.d = np.ascontiguousarray(d, dtype=np.int32)
        self.p = np.ascontiguousarray(p, dtype=np.int32)
        self.n = int(self.p.shape[0])
        assert self.d.shape == (self.n + 1, self.n + 1)
        self.m, self.R, self.Q = int(m), int(R), int(Q)
        self.flags = LOAD_FULL if load_full else 0
        self.c = Inst(self.n, self.m, self.R, self.Q, self.flags, _p(self.d), _p(self.p))

    @classmethod
    def from_workload(cls, inst, load_full=False):
        return cls(euc2d(inst.coords), inst.p, inst.m, inst.R, inst.Q, load_full)


def evaluate(I, ops, off, allow_partial=False, with_times=False):
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    z = np.zeros(1, np.int32)
    st = np.zeros(1, np.uint32)
    times = np.zeros(2 * I.n + 2, np.int64) if with_times else None
    rc = lib().oracle_evaluate(C.byref(I.c), _p(ops), _p(off), int(allow_partial), _p(z),
                               _p(st, C.c_uint32), _p(times, C.c_int64) if with_times else None)
    if rc != 0:
        raise OverflowError("oracle: a time exceeded int32")
    if with_times:
        return int(z[0]), int(st[0]), times
    return int(z[0]), int(st[0])


def evaluate_batch(I, ops, off, threads=1):
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    count = ops.shape[0]
    z = np.zeros(count, np.int32)
    st = np.zeros(count, np.uint32)
    lib().oracle_evaluate_batch(C.byref(I.c), count, _p(ops), _p(off), _p(z), _p(st, C.c_uint32),
                                threads)
    return z, st


def sp_closure(d):
    d = np.ascontiguousarray(d, dtype=np.int32)
    N = d.shape[0]
    sp = np.empty((N, N), np.int64)
    lib().oracle_sp_closure(_p(d), N, _p(sp, C.c_int64))
    return sp


def bruteforce(I):
    ops = np.zeros(2 * I.n, np.int32)
    off = np.zeros(I.m + 1, np.int32)
    best = lib().oracle_bruteforce(C.byref(I.c), _p(ops), _p(off))
    return int(best), ops, off


def minmax_vrp(d, n, m):
    d = np.ascontiguousarray(d, dtype=np.int32)
    return int(lib().oracle_minmax_vrp(_p(d), n, m))


def held_karp(d, n):
    d = np.ascontiguousarray(d, dtype=np.int32)
    return int(lib().oracle_held_karp(_p(d), n))


def splitmix64_stream(seed, count):
    s = C.c_uint64(seed)
    return [int(lib().oracle_splitmix64_next(C.byref(s))) for _ in range(count)]


def rng(key, counter):
    return int(lib().oracle_rng(C.c_uint64(key), C.c_uint64(counter)))


def exp(x):
    return float(lib().oracle_exp(float(x)))


def q_range(n):
    a = np.zeros(1, np.int32)
    b = np.zeros(1, np.int32)
    lib().oracle_q_range(n, _p(a), _p(b))
    return int(a[0]), int(b[0])


def insertion_matrix(I, ops, off, c):
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    G = int(off[-1]) + I.m
    out = np.zeros((G, G), np.int32)
    trav = np.zeros((G, G), np.int32)
    st = np.zeros((G, G), np.uint32)
    rc = lib().oracle_insertion_matrix(C.byref(I.c), _p(ops), _p(off), int(c), _p(out), _p(trav),
                                       _p(st, C.c_uint32))
    if rc != 0:
        raise ValueError("oracle_insertion_matrix failed")
    return out, trav, st


def initial_solution(I, coords):
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    ops = np.zeros(2 * I.n, np.int32)
    off = np.zeros(I.m + 1, np.int32)
    rc = lib().oracle_initial_solution(C.byref(I.c), _p(coords), _p(ops), _p(off))
    if rc != 0:
        raise ValueError("oracle_initial_solution failed")
    return ops, off


def alns_params(iterations, q_min=0, q_max=0, repair_mask=3, destroy_mask=1, ls_pickup_every=200,
                ls_relocate_every=500):
    return AlnsParams(0.30, 0.9998, 0.50, 0.1, 2000, 100, 33, 9, 13, 0.1, q_min, q_max,
                      iterations, repair_mask, destroy_mask, ls_pickup_every, ls_relocate_every)


def alns_run(I, init_ops, init_off, params, seed):
    init_ops = np.ascontiguousarray(init_ops, dtype=np.int32)
    init_off = np.ascontiguousarray(init_off, dtype=np.int32)
    bo = np.zeros(2 * I.n, np.int32)
    bf = np.zeros(I.m + 1, np.int32)
    co = np.zeros(2 * I.n, np.int32)
    cf = np.zeros(I.m + 1, np.int32)
    st = AlnsStats()
    trace = np.zeros(max(1, params.iterations), np.int32)
    rc = lib().oracle_alns_run(C.byref(I.c), _p(init_ops), _p(init_off), C.byref(params),
                               C.c_uint64(seed), _p(bo), _p(bf), _p(co), _p(cf), C.byref(st),
                               _p(trace))
    if rc != 0:
        raise ValueError(f"oracle_alns_run failed rc={rc}")
    return dict(best_ops=bo, best_off=bf, cur_ops=co, cur_off=cf, stats=st, trace=trace)


def decode(I, keys, layout=LAYOUT_VKEYS):
    keys = np.ascontiguousarray(keys, dtype=np.float32)
    assert keys.shape[-1] == key_length(I, layout)
    ops = np.zeros(2 * I.n, np.int32)
    off = np.zeros(I.m + 1, np.int32)
    z = np.zeros(1, np.int32)
    un = np.zeros(1, np.int32)
    fit = np.zeros(1, np.int64)
    lib().oracle_decode_l(C.byref(I.c), _p(keys, C.c_float), layout, _p(ops), _p(off), _p(z), _p(un),
                          _p(fit, C.c_int64))
    return ops, off, int(z[0]), int(un[0]), int(fit[0])


def encode(I, ops, off, layout=LAYOUT_VKEYS):
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    keys = np.zeros(key_length(I, layout), np.float32)
    lib().oracle_encode_l(C.byref(I.c), _p(ops), _p(off), layout, _p(keys, C.c_float))
    return keys


def brkga_params(pop, generations, elite=0.2, mutant=0.1, rho=0.7, warm_frac=0.15,
                 warm_variants=20, eps=0.03, layout=LAYOUT_VKEYS):
    import math
    return BrkgaParams(pop, generations, int(math.ceil(warm_frac * pop - 1e-9)), warm_variants,
                       elite, mutant, rho, eps, layout)


def brkga_run(I, params, warm_ops, warm_off, seed):
    L = key_length(I, params.layout)
    keys = np.zeros((params.pop, L), np.float32)
    trace = np.zeros(max(1, params.generations), np.int64)
    bo = np.zeros(2 * I.n, np.int32)
    bf = np.zeros(I.m + 1, np.int32)
    best = np.zeros(1, np.int64)
    wo = None if warm_ops is None else np.ascontiguousarray(warm_ops, dtype=np.int32)
    wf = None if warm_off is None else np.ascontiguousarray(warm_off, dtype=np.int32)
    rc = lib().oracle_brkga_run(C.byref(I.c), C.byref(params), _p(wo) if wo is not None else None,
                                _p(wf) if wf is not None else None, C.c_uint64(seed),
                                _p(keys, C.c_float), _p(trace, C.c_int64), _p(bo), _p(bf),
                                _p(best, C.c_int64))
    if rc != 0:
        raise ValueError(f"oracle_brkga_run failed rc={rc}")
    return dict(keys=keys, trace=trace, best_ops=bo, best_off=bf, best_fitness=int(best[0]))


DESTROY = {"random": 0, "worst": 1, "shaw": 2, "cluster": 3, "route": 4, "critical": 5}


def coordination(I, ops, off):
    """Section 5.2 counts of one complete solution: (cross, interleaved, status);
    -1 where a count is undefined (malformed; interleaved on a cycle)."""
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    cr = np.zeros(1, np.int32)
    il = np.zeros(1, np.int32)
    st = lib().oracle_coordination(C.byref(I.c), _p(ops), _p(off), _p(cr), _p(il))
    return int(cr[0]), int(il[0]), int(st)


def alns_run_replicas(I, init_ops, init_off, params, seed, replicas, sync_every=1000):
    """R replicas of Algorithm 1 with the best-of-all import every sync_every
    iterations (Section 4.2.1)."""
    init_ops = np.ascontiguousarray(init_ops, dtype=np.int32)
    init_off = np.ascontiguousarray(init_off, dtype=np.int32)
    bo = np.zeros(2 * I.n, np.int32)
    bf = np.zeros(I.m + 1, np.int32)
    br = np.zeros(1, np.int32)
    imp = np.zeros(1, np.int32)
    stats = (AlnsStats * replicas)()
    traces = np.zeros((replicas, max(1, params.iterations)), np.int32)
    rc = lib().oracle_alns_run_replicas(C.byref(I.c), _p(init_ops), _p(init_off), C.byref(params),
                                        C.c_uint64(seed), replicas, sync_every, _p(bo), _p(bf), _p(br),
                                        stats, _p(traces), _p(imp))
    if rc != 0:
        raise ValueError(f"oracle_alns_run_replicas failed rc={rc}")
    return dict(best_ops=bo, best_off=bf, best_replica=int(br[0]), stats=list(stats),
                traces=traces[:, :params.iterations], imports=int(imp[0]))


def initial_solution_paper(I, coords, refine_rounds=10):
    """The paper's three-phase constructor and its refinement (Section 4.2.5)."""
    ops = np.zeros(2 * I.n, np.int32)
    off = np.zeros(I.m + 1, np.int32)
    cc = np.ascontiguousarray(coords, dtype=np.int32) if coords is not None else None
    rc = lib().oracle_initial_solution_paper(C.byref(I.c), _p(cc) if cc is not None else None, refine_rounds,
                                             _p(ops), _p(off))
    if rc != 0:
        raise ValueError(f"oracle_initial_solution_paper failed rc={rc}")
    return ops, off


LS_PICKUP, LS_RELOCATE = 1, 2


def local_search(I, mode, ops, off, passes=3):
    """Section 4.2.6 local search on a copy of (ops, off): (moves, z, ops, off)."""
    ops = np.array(ops, dtype=np.int32)
    off = np.array(off, dtype=np.int32)
    z = np.zeros(1, np.int32)
    mv = lib().oracle_local_search(C.byref(I.c), mode, passes, _p(ops), _p(off), _p(z))
    if mv < 0:
        raise ValueError("local search needs a feasible complete solution and mode 1 or 2")
    return mv, int(z[0]), ops, off


SEED_NN, SEED_LB, SEED_SPT = 0, 1, 2


def seed_chromosome(I, h, layout=LAYOUT_VKEYS):
    """Construction seed h of the BRKGA warm start (Section 4.4.4)."""
    keys = np.zeros(key_length(I, layout), np.float32)
    lib().oracle_seed_chromosome(C.byref(I.c), h, layout, _p(keys, C.c_float))
    return keys


def destroy(I, op, ops, off, q, qmin, key, base):
    """One destroy step on (ops, off); returns the boolean removal mask over customers 0..n."""
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    rem = C.create_string_buffer(I.n + 1)
    cnt = lib().oracle_destroy(C.byref(I.c), DESTROY.get(op, op), _p(ops), _p(off), q, qmin,
                               C.c_uint64(key), C.c_uint64(base), rem)
    mask = np.frombuffer(rem.raw, dtype=np.uint8).astype(bool)
    assert int(mask.sum()) == cnt
    return mask


REPAIR = {"greedy": 0, "regret2": 1, "regret3": 2, "regretm": 3}


def repair(I, op, ops, off, removed, max_steps=-1):
    """The repair operator op (Section 4.2.3) on a partial solution: reinsert
    the customers `removed` (at most max_steps insertions); returns (ops, off)
    or None when some customer has no feasible insertion."""
    ops = np.ascontiguousarray(ops if len(ops) else np.zeros(1, np.int32), dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    rem = np.ascontiguousarray(sorted(int(c) for c in removed), dtype=np.int32)
    N = int(off[-1])
    oo = np.zeros(N + 2 * len(rem) + 1, np.int32)
    of = np.zeros(I.m + 1, np.int32)
    rc = lib().oracle_repair(C.byref(I.c), REPAIR.get(op, op), _p(ops), _p(off),
                             _p(rem if len(rem) else np.zeros(1, np.int32)), len(rem), max_steps, _p(oo), _p(of))
    if rc != 0:
        return None
    return oo[:int(of[-1])].copy(), of


def alns_adapt_script(params, z0, steps):
    """Algorithm 1's acceptance and adaptation on scripted iterations: steps is
    a list of (destroy op, repair op, candidate makespan, status, SA draw u).
    Returns (stats, z_trace)."""
    k = len(steps)
    di = np.array([s[0] for s in steps] or [0], np.int32)
    rj = np.array([s[1] for s in steps] or [0], np.int32)
    zn = np.array([s[2] for s in steps] or [0], np.int32)
    st = np.array([s[3] for s in steps] or [0], np.uint32)
    u = np.array([s[4] for s in steps] or [0.0], np.float64)
    stats = AlnsStats()
    trace = np.zeros(max(1, k), np.int32)
    rc = lib().oracle_alns_adapt_script(C.byref(params), int(z0), k, _p(di), _p(rj), _p(zn), _p(st, C.c_uint32),
                                        _p(u, C.c_double), C.byref(stats), _p(trace))
    if rc != 0:
        raise ValueError("bad operator index in the script")
    return stats, trace[:k]
