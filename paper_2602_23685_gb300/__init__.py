"""Python binding of libvrprpd (argument marshalling only).

Every computation runs in the CUDA library declared in include/vrprpd.h; this
module passes device pointers (from torch tensors), sizes and the current
torch stream through ctypes.  There is no fallback: if the library or a CUDA
device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB, build as _build

__all__ = ["lib", "Instance", "evaluate", "evaluate_host", "evaluate_plain", "autotune",
           "set_eval_config", "get_eval_config", "sync", "VrpError",
           "CYCLE", "VEH_CAP", "POOL", "MALFORMED", "DIST_MODES"]

CYCLE, VEH_CAP, POOL, MALFORMED = 1, 2, 4, 8
LOAD_MIN, LOAD_FULL = 0, 1
DIST_MODES = {"auto": 0, "smem32": 1, "smem16": 2, "global16": 3, "global32": 4, "coords": 5}
_DIST_NAMES = {v: k for k, v in DIST_MODES.items()}
INT32_MAX = 2**31 - 1

_lock = threading.Lock()
_lib = None


class VrpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libvrprpd error {code}: {msg}")
        self.code = code


class Batch(C.Structure):
    _fields_ = [("num", C.c_int32), ("ops", C.c_void_p), ("off", C.c_void_p)]


class EvalConfig(C.Structure):
    _fields_ = [("dist_mode", C.c_int32), ("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("walk", C.c_int32), ("group_warps", C.c_int32)]


WALKS = {"staged": 0, "streamed": 1}
_WALK_NAMES = {v: k for k, v in WALKS.items()}


def lib():
    """Load (building first if needed) the in-tree libvrprpd.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = LIB if os.path.exists(LIB) else _build()
            L = C.CDLL(path)
            vp, i32, u32 = C.c_void_p, C.c_int32, C.c_uint32
            L.vrprpd_instance_create.argtypes = [vp, vp, i32, i32, i32, i32, u32, C.POINTER(vp)]
            L.vrprpd_instance_create_dist.argtypes = [vp, vp, i32, i32, i32, i32, u32, C.POINTER(vp)]
            L.vrprpd_instance_destroy.argtypes = [vp]
            L.vrprpd_instance_destroy.restype = None
            L.vrprpd_instance_get_dist.argtypes = [vp, vp]
            # vrprpd_batch16 has vrprpd_batch's layout (int32, two pointers)
            for name in ("vrprpd_evaluate", "vrprpd_evaluate_host", "vrprpd_evaluate_plain", "vrprpd_coordination",
                         "vrprpd_evaluate16", "vrprpd_evaluate16_host"):
                getattr(L, name).argtypes = [vp, C.POINTER(Batch), vp, vp, vp]
            L.vrprpd_sync.argtypes = [vp, vp]
            L.vrprpd_eval_set_config.argtypes = [vp, C.POINTER(EvalConfig)]
            L.vrprpd_eval_get_config.argtypes = [vp, C.POINTER(EvalConfig)]
            L.vrprpd_autotune.argtypes = [vp, C.POINTER(Batch), vp, C.POINTER(EvalConfig)]
            L.vrprpd_last_error.restype = C.c_char_p
            _register_extra(L)
            _lib = L
    return _lib


def _register_extra(L):
    """Signatures of the search entry points (declared in include/vrprpd.h)."""
    from . import _search_sig
    _search_sig.register(L)


def _check(rc):
    if rc != 0:
        raise VrpError(rc, lib().vrprpd_last_error().decode(errors="replace"))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libvrprpd needs a CUDA device; none is available")
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _is16(dtype):
    """True for a 16-bit integer dtype (torch or numpy)."""
    import torch
    if isinstance(dtype, torch.dtype):
        return dtype == torch.int16 or dtype == getattr(torch, "uint16", torch.int16)
    return np.dtype(dtype) in (np.dtype(np.int16), np.dtype(np.uint16))


def _dev_i32(t, name, shape=None, wide16=False):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or \
            not (t.dtype == torch.int32 or (wide16 and _is16(t.dtype))):
        raise TypeError(f"{name} must be a CUDA int32 tensor" + (" (or int16 for ops and off both)" if wide16 else ""))
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


class Instance:
    """A VRP-RPD instance resident on the current CUDA device."""

    def __init__(self, m, R, Q, p, coords=None, d=None, load_full=False):
        L = lib()
        _torch()
        p = np.ascontiguousarray(p, dtype=np.int32)
        self.n = int(p.shape[0])
        self.m, self.R, self.Q = int(m), int(R), int(Q)
        self.load_full = bool(load_full)
        flags = LOAD_FULL if load_full else LOAD_MIN
        h = C.c_void_p()
        if coords is not None:
            coords = np.ascontiguousarray(coords, dtype=np.int32)
            if coords.shape != (self.n + 1, 2):
                raise ValueError("coords must be (n+1) x 2")
            _check(L.vrprpd_instance_create(coords.ctypes.data, p.ctypes.data, self.n, self.m,
                                            self.R, self.Q, flags, C.byref(h)))
        elif d is not None:
            d = np.ascontiguousarray(d, dtype=np.int32)
            if d.shape != (self.n + 1, self.n + 1):
                raise ValueError("d must be (n+1) x (n+1)")
            _check(L.vrprpd_instance_create_dist(d.ctypes.data, p.ctypes.data, self.n, self.m,
                                                 self.R, self.Q, flags, C.byref(h)))
        else:
            raise ValueError("need coords or d")
        self._h = h
        self.p = p
        self.coords = coords

    @classmethod
    def from_workload(cls, w, load_full=False):
        return cls(w.m, w.R, w.Q, w.p, coords=w.coords, load_full=load_full)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("instance closed")
        return self._h

    def dist(self):
        d = np.empty((self.n + 1, self.n + 1), np.int32)
        _check(lib().vrprpd_instance_get_dist(self.handle, d.ctypes.data))
        return d

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().vrprpd_instance_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch(inst, ops, off, wide16=False):
    B = ops.shape[0]
    _dev_i32(ops, "ops", (B, 2 * inst.n), wide16)
    _dev_i32(off, "off", (B, inst.m + 1), wide16)
    if _is16(ops.dtype) != _is16(off.dtype):
        raise TypeError("ops and off must both be 32-bit or both 16-bit")
    return Batch(B, ops.data_ptr(), off.data_ptr())


def evaluate(inst, ops, off, z=None, st=None, stream=None):
    """Batched evaluation on device tensors; returns (makespan int32, status int32 view).
    ops and off are int32, or both int16 (the 16-bit form: the same codes in half the bytes)."""
    torch = _torch()
    b = _batch(inst, ops, off, wide16=True)
    if z is None:
        z = torch.empty(b.num, dtype=torch.int32, device=ops.device)
    if st is None:
        st = torch.empty(b.num, dtype=torch.int32, device=ops.device)
    fn = lib().vrprpd_evaluate16 if _is16(ops.dtype) else lib().vrprpd_evaluate
    _check(fn(inst.handle, C.byref(b), z.data_ptr(), st.data_ptr(), _stream_ptr(stream)))
    return z, st


def evaluate_plain(inst, ops, off, z=None, st=None, stream=None):
    """The plain one-thread-per-candidate GPU form (comparison baseline)."""
    torch = _torch()
    b = _batch(inst, ops, off)
    if z is None:
        z = torch.empty(b.num, dtype=torch.int32, device=ops.device)
    if st is None:
        st = torch.empty(b.num, dtype=torch.int32, device=ops.device)
    _check(lib().vrprpd_evaluate_plain(inst.handle, C.byref(b), z.data_ptr(), st.data_ptr(),
                                       _stream_ptr(stream)))
    return z, st


def coordination(inst, ops, off, stream=None):
    """Section 5.2 counts of complete solutions on device tensors: (cross,
    interleaved) int32 per candidate, -1 where undefined."""
    torch = _torch()
    b = _batch(inst, ops, off)
    cross = torch.empty(b.num, dtype=torch.int32, device=ops.device)
    inter = torch.empty(b.num, dtype=torch.int32, device=ops.device)
    _check(lib().vrprpd_coordination(inst.handle, C.byref(b), cross.data_ptr(), inter.data_ptr(),
                                     _stream_ptr(stream)))
    return cross, inter


def evaluate_host(inst, ops, off, z=None, st=None, stream=None):
    """Evaluation from host memory (numpy arrays or CPU tensors; pinned tensors are
    read in place, others copied in), returning when done.  ops and off are int32,
    or both 16-bit (the same codes in half the bytes across the host link)."""
    wide = _is16(ops.dtype)

    def host_ptr(a, name, operand=True):
        if hasattr(a, "data_ptr"):
            if a.device.type != "cpu" or not a.is_contiguous():
                raise TypeError(f"{name} must be a contiguous CPU tensor")
            if operand and _is16(a.dtype) != wide:
                raise TypeError("ops and off must both be 32-bit or both 16-bit")
            if operand and not wide and a.dtype != _torch().int32:
                raise TypeError(f"{name} must be int32 or 16-bit")
            return a.data_ptr()
        ok = isinstance(a, np.ndarray) and a.flags.c_contiguous and \
            (not operand or (a.dtype in (np.int16, np.uint16)) == wide and (wide or a.dtype == np.int32))
        if not ok:
            raise TypeError(f"{name} must be a contiguous array: int32, or 16-bit for ops and off both")
        return a.ctypes.data
    B = ops.shape[0]
    if tuple(ops.shape) != (B, 2 * inst.n) or tuple(off.shape) != (B, inst.m + 1):
        raise ValueError("bad ops/off shape")
    if z is None:
        z = np.empty(B, np.int32)
    if st is None:
        st = np.empty(B, np.uint32)
    b = Batch(B, host_ptr(ops, "ops"), host_ptr(off, "off"))
    fn = lib().vrprpd_evaluate16_host if wide else lib().vrprpd_evaluate_host
    _check(fn(inst.handle, C.byref(b), host_ptr(z, "z", False) if hasattr(z, "data_ptr") else z.ctypes.data,
              st.data_ptr() if hasattr(st, "data_ptr") else st.ctypes.data, _stream_ptr(stream)))
    return z, st


def sync(inst, stream=None):
    _check(lib().vrprpd_sync(inst.handle, _stream_ptr(stream)))


def set_eval_config(inst, dist_mode="auto", warps_per_block=0, blocks_per_sm=0, walk="staged", group_warps=1):
    cfg = EvalConfig(DIST_MODES[dist_mode] if isinstance(dist_mode, str) else int(dist_mode),
                     warps_per_block, blocks_per_sm, WALKS[walk] if isinstance(walk, str) else int(walk),
                     group_warps)
    _check(lib().vrprpd_eval_set_config(inst.handle, C.byref(cfg)))


def _cfg_dict(cfg):
    return {"dist_mode": _DIST_NAMES[cfg.dist_mode], "warps_per_block": cfg.warps_per_block,
            "blocks_per_sm": cfg.blocks_per_sm, "walk": _WALK_NAMES.get(cfg.walk, cfg.walk),
            "group_warps": cfg.group_warps}


def get_eval_config(inst):
    cfg = EvalConfig()
    _check(lib().vrprpd_eval_get_config(inst.handle, C.byref(cfg)))
    return _cfg_dict(cfg)


def autotune(inst, ops, off, stream=None):
    b = _batch(inst, ops, off)
    cfg = EvalConfig()
    _check(lib().vrprpd_autotune(inst.handle, C.byref(b), _stream_ptr(stream), C.byref(cfg)))
    return _cfg_dict(cfg)


# ---------------------------------------------------------------------------
# ALNS (Section 4.2)
# ---------------------------------------------------------------------------
def _sol(inst, ops=None, off=None):
    from ._search_sig import Solution
    ops = np.zeros(2 * inst.n, np.int32) if ops is None else np.ascontiguousarray(ops, dtype=np.int32)
    off = np.zeros(inst.m + 1, np.int32) if off is None else np.ascontiguousarray(off, dtype=np.int32)
    return Solution(ops.ctypes.data, off.ctypes.data, 0, 0), ops, off


def initial_solution(inst):
    s, ops, off = _sol(inst)
    _check(lib().vrprpd_initial_solution(inst.handle, C.byref(s)))
    return ops, off


def initial_solution_paper(inst, refine_rounds=10, stream=None):
    """The paper's three-phase constructor and its refinement (Section 4.2.5),
    on the device; returns (ops, off, makespan)."""
    s, ops, off = _sol(inst)
    _check(lib().vrprpd_initial_solution_paper(inst.handle, refine_rounds, C.byref(s), _stream_ptr(stream)))
    return ops, off, s.makespan


def alns_params(iterations=1000, q_min=0, q_max=0, repair_mask=3, team_blocks=0, **over):
    from ._search_sig import AlnsParams
    p = AlnsParams()
    lib().vrprpd_alns_params_default(C.byref(p))
    p.iterations, p.q_min, p.q_max = iterations, q_min, q_max
    p.repair_mask, p.team_blocks = repair_mask, team_blocks
    for k, v in over.items():
        setattr(p, k, v)
    return p


def alns_run(inst, params, seed=0, init=None, stream=None):
    """Algorithm 1 on the device.  init = (ops, off) host arrays or None."""
    from ._search_sig import AlnsStats
    best, bo, bf = _sol(inst)
    cur, co, cf = _sol(inst)
    init_s = None
    if init is not None:
        init_s, _io, _if = _sol(inst, *init)
    st = AlnsStats()
    R = max(1, params.replicas)
    traces = np.zeros((R, max(1, params.iterations)), np.int32)
    _check(lib().vrprpd_alns_run(inst.handle, C.byref(init_s) if init_s is not None else None, C.byref(params),
                                 C.c_uint64(seed), C.byref(best), C.byref(cur), C.byref(st),
                                 traces.ctypes.data, _stream_ptr(stream)))
    return {"best_ops": bo, "best_off": bf, "z_best": best.makespan, "cur_ops": co, "cur_off": cf,
            "z_current": cur.makespan, "stats": st, "trace": traces[0, :params.iterations],
            "traces": traces[:, :params.iterations]}


def insertion_matrix(inst, ops, off, c, stream=None):
    """Full insertion-delta matrix of customer c into a host partial solution."""
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    G = int(off[-1]) + inst.m
    delta = np.empty((G, G), np.int32)
    travel = np.empty((G, G), np.int32)
    opsp = ops if ops.size else np.zeros(1, np.int32)
    _check(lib().vrprpd_insertion_matrix(inst.handle, opsp.ctypes.data, off.ctypes.data, int(c),
                                         delta.ctypes.data, travel.ctypes.data, _stream_ptr(stream)))
    return delta, travel


def repair_then_matrix(inst, ops, off, removed, steps, repair_op=0, team_blocks=0, stream=None):
    """`steps` repair insertions of the customers `removed` into the host
    partial solution (ops, off), then the insertion-delta matrix of the
    smallest customer still to insert.  Returns (ops, off, delta, travel,
    incremental steps)."""
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int32)
    rem = np.ascontiguousarray(sorted(int(c) for c in removed), dtype=np.int32)
    nout = int(off[-1]) + 2 * int(steps)
    G = nout + inst.m
    oo = np.zeros(max(nout, 1), np.int32)
    of = np.zeros(inst.m + 1, np.int32)
    delta = np.empty((G, G), np.int32)
    travel = np.empty((G, G), np.int32)
    inc = np.zeros(1, np.int64)
    opsp = ops if ops.size else np.zeros(1, np.int32)
    _check(lib().vrprpd_repair_then_matrix(inst.handle, opsp.ctypes.data, off.ctypes.data, rem.ctypes.data,
                                           len(rem), int(repair_op), int(steps), int(team_blocks), oo.ctypes.data,
                                           of.ctypes.data, delta.ctypes.data, travel.ctypes.data, inc.ctypes.data,
                                           _stream_ptr(stream)))
    return oo[:nout], of, delta, travel, int(inc[0])


# ---------------------------------------------------------------------------
# BRKGA (Section 4.4)
# ---------------------------------------------------------------------------
LAYOUT_VKEYS = 0   # 2n op priorities + m vehicle keys
LAYOUT_HINTS = 1   # 2n op priorities + 2n assignment hints (the paper's 4n chromosome)


def key_length(inst, layout=LAYOUT_VKEYS):
    return 4 * inst.n if layout == LAYOUT_HINTS else 2 * inst.n + inst.m


def brkga_params(pop, generations, elite=0.2, mutant=0.1, rho=0.7, warm_slots=-1, warm_variants=20,
                 eps=0.03, layout=LAYOUT_VKEYS):
    """BRKGA parameters; warm_slots=-1 lets the library seed ceil(0.15 pop)
    slots from the warm start (Section 4.4.4)."""
    from ._search_sig import BrkgaParams
    return BrkgaParams(pop, generations, warm_slots, warm_variants,
                       elite, mutant, rho, eps, layout)


def brkga_decode(inst, keys, layout=LAYOUT_VKEYS, stream=None):
    """Decode device keys (num x L float32, L by layout) -> routes, makespan, unscheduled, fitness."""
    torch = _torch()
    if keys.dtype != torch.float32 or keys.device.type != "cuda" or not keys.is_contiguous():
        raise TypeError("keys must be a contiguous CUDA float32 tensor")
    num = keys.shape[0]
    if tuple(keys.shape) != (num, key_length(inst, layout)):
        raise ValueError(f"keys must be num x {key_length(inst, layout)}")
    dev = keys.device
    ops = torch.empty((num, 2 * inst.n), dtype=torch.int32, device=dev)
    off = torch.empty((num, inst.m + 1), dtype=torch.int32, device=dev)
    z = torch.empty(num, dtype=torch.int32, device=dev)
    un = torch.empty(num, dtype=torch.int32, device=dev)
    fit = torch.empty(num, dtype=torch.int64, device=dev)
    _check(lib().vrprpd_brkga_decode(inst.handle, keys.data_ptr(), num, layout, ops.data_ptr(), off.data_ptr(),
                                     z.data_ptr(), un.data_ptr(), fit.data_ptr(), _stream_ptr(stream)))
    return ops, off, z, un, fit


def brkga_run(inst, params, seed=0, warm=None, final_keys=False, stream=None):
    """Warm-started BRKGA on the device; warm = (ops, off) host arrays or None."""
    torch = _torch()
    best, bo, bf = _sol(inst)
    warm_s = None
    if warm is not None:
        warm_s, _wo, _wf = _sol(inst, *warm)
    trace = np.zeros(params.generations, np.int64)
    fitness = np.zeros(1, np.int64)
    keys = None
    if final_keys:
        keys = torch.empty((params.pop, key_length(inst, params.layout)), dtype=torch.float32, device="cuda")
    _check(lib().vrprpd_brkga_run(inst.handle, C.byref(params), C.byref(warm_s) if warm_s is not None else None,
                                  C.c_uint64(seed), C.byref(best), fitness.ctypes.data, trace.ctypes.data,
                                  keys.data_ptr() if keys is not None else None, _stream_ptr(stream)))
    return {"best_ops": bo, "best_off": bf, "z_best": best.makespan, "best_fitness": int(fitness[0]),
            "trace": trace, "keys": keys}


# ---------------------------------------------------------------------------
# many instances in one persistent launch
# ---------------------------------------------------------------------------
class MultiBatch:
    """A plan over (instance, ops, off) triples of uneven size; evaluate() runs
    them all in one persistent launch (replayed as a CUDA graph)."""

    def __init__(self, items):
        torch = _torch()
        L = lib()
        self.items = list(items)
        n = len(self.items)
        self.z = [torch.empty(ops.shape[0], dtype=torch.int32, device=ops.device) for _, ops, _ in self.items]
        self.st = [torch.empty(ops.shape[0], dtype=torch.int32, device=ops.device) for _, ops, _ in self.items]
        self._insts = (C.c_void_p * n)(*[inst.handle.value for inst, _, _ in self.items])
        self._batches = (Batch * n)(*[_batch(inst, ops, off) for inst, ops, off in self.items])
        self._z = (C.c_void_p * n)(*[t.data_ptr() for t in self.z])
        self._st = (C.c_void_p * n)(*[t.data_ptr() for t in self.st])
        h = C.c_void_p()
        _check(L.vrprpd_multi_create(C.cast(self._insts, C.c_void_p), C.cast(self._batches, C.c_void_p),
                                     C.cast(self._z, C.c_void_p), C.cast(self._st, C.c_void_p), n, C.byref(h)))
        self._h = h

    def evaluate(self, stream=None):
        _check(lib().vrprpd_multi_evaluate(self._h, _stream_ptr(stream)))
        return self.z, self.st

    def autotune(self, stream=None):
        cfg = EvalConfig()
        _check(lib().vrprpd_multi_autotune(self._h, _stream_ptr(stream), C.byref(cfg)))
        return _cfg_dict(cfg)

    def set_config(self, dist_mode="global16", warps_per_block=8, walk="staged"):
        cfg = EvalConfig(DIST_MODES[dist_mode], warps_per_block, 0, WALKS[walk], 1)
        _check(lib().vrprpd_multi_set_config(self._h, C.byref(cfg)))

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().vrprpd_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
class Server:
    """Continuous-batching solve server (vrprpd_server_*): requests are admitted
    by memory budget and worker slots and run concurrently on the device."""

    def __init__(self, mem_budget_bytes, max_active=4):
        L = lib()
        _torch()
        h = C.c_void_p()
        _check(L.vrprpd_server_create(C.c_size_t(int(mem_budget_bytes)), int(max_active), C.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, w, alns_iterations, brkga_pop=0, brkga_generations=0, seed=0, q_min=0, q_max=0, **alns_over):
        """alns_over: further vrprpd_alns_params fields (init_mode, init_refine_rounds, ...)."""
        from ._search_sig import Request
        coords = np.ascontiguousarray(w.coords, dtype=np.int32)
        p = np.ascontiguousarray(w.p, dtype=np.int32)
        req = Request(coords.ctypes.data, p.ctypes.data, w.n, w.m, w.R, w.Q, 0,
                      alns_params(alns_iterations, q_min, q_max, **alns_over),
                      brkga_params(max(brkga_pop, 2), brkga_generations), C.c_uint64(seed))
        rid = C.c_int64()
        _check(lib().vrprpd_server_submit(self._h, C.byref(req), C.byref(rid)))
        self._keep[rid.value] = (w.n, w.m)
        return rid.value

    def _result(self, fn, rid):
        from ._search_sig import Result
        n, m = self._keep[rid]
        res = Result()
        ops = np.zeros(2 * n, np.int32)
        off = np.zeros(m + 1, np.int32)
        rc = fn(self._h, C.c_int64(rid), C.byref(res), ops.ctypes.data, off.ctypes.data)
        if rc == -6:
            return None
        _check(rc)
        return {"id": res.id, "status": res.status, "z_alns": res.z_alns, "z_brkga": res.z_brkga,
                "z_best": res.z_best, "ops": ops, "off": off, "t_submit_ms": res.t_submit_ms,
                "t_start_ms": res.t_start_ms, "t_end_ms": res.t_end_ms, "device_ms": res.device_ms,
                "message": res.message.decode(errors="replace")}

    def poll(self, rid):
        return self._result(lib().vrprpd_server_poll, rid)

    def wait(self, rid):
        return self._result(lib().vrprpd_server_wait, rid)

    def stats(self):
        from ._search_sig import ServerStats
        st = ServerStats()
        _check(lib().vrprpd_server_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def cancel_pending(self):
        """Withdraw the requests not admitted yet; returns how many."""
        k = np.zeros(1, np.int32)
        _check(lib().vrprpd_server_cancel_pending(self._h, k.ctypes.data))
        return int(k[0])

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().vrprpd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
