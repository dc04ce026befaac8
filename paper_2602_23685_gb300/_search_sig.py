"""ctypes declarations of the search entry points (include/vrprpd.h)."""
import ctypes as C


class Solution(C.Structure):
    _fields_ = [("ops", C.c_void_p), ("off", C.c_void_p), ("makespan", C.c_int32), ("status", C.c_uint32)]


class AlnsParams(C.Structure):
    _fields_ = [("T0", C.c_double), ("alpha", C.c_double), ("reheat", C.c_double), ("r", C.c_double),
                ("stagnation", C.c_int32), ("tau", C.c_int32), ("sigma1", C.c_int32),
                ("sigma2", C.c_int32), ("sigma3", C.c_int32), ("w_min", C.c_double),
                ("q_min", C.c_int32), ("q_max", C.c_int32), ("iterations", C.c_int32),
                ("repair_mask", C.c_int32), ("team_blocks", C.c_int32),
                ("destroy_mask", C.c_int32), ("ls_pickup_every", C.c_int32), ("ls_relocate_every", C.c_int32),
                ("replicas", C.c_int32), ("sync_every", C.c_int32), ("init_mode", C.c_int32),
                ("init_refine_rounds", C.c_int32), ("wait_limit_ns", C.c_int64)]


class AlnsStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accepted", C.c_int32), ("improved", C.c_int32),
                ("new_best", C.c_int32), ("reheats", C.c_int32), ("rejected_infeasible", C.c_int32),
                ("z_init", C.c_int32), ("z_best", C.c_int32), ("z_current", C.c_int32),
                ("T_final", C.c_double), ("w_destroy", C.c_double * 8), ("w_repair", C.c_double * 4),
                ("device_ms", C.c_double), ("matrix_entries", C.c_int64),
                ("fallback_entries", C.c_int64), ("team_blocks", C.c_int32), ("phase_ms", C.c_double * 6),
                ("incremental_steps", C.c_int64), ("full_steps", C.c_int64), ("ls_moves", C.c_int32),
                ("ls_new_best", C.c_int32), ("ls_ms", C.c_double), ("replicas", C.c_int32),
                ("imports", C.c_int32), ("best_replica", C.c_int32), ("pruned_entries", C.c_int64),
                ("tiles", C.c_int64), ("tiles_pruned", C.c_int64)]


class BrkgaParams(C.Structure):
    _fields_ = [("pop", C.c_int32), ("generations", C.c_int32), ("warm_slots", C.c_int32),
                ("warm_variants", C.c_int32), ("elite_frac", C.c_float), ("mutant_frac", C.c_float),
                ("rho", C.c_float), ("eps", C.c_float), ("layout", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("coords", C.c_void_p), ("p", C.c_void_p), ("n", C.c_int32), ("m", C.c_int32),
                ("R", C.c_int32), ("Q", C.c_int32), ("flags", C.c_uint32), ("alns", AlnsParams),
                ("brkga", BrkgaParams), ("seed", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("z_alns", C.c_int32), ("z_brkga", C.c_int32),
                ("z_best", C.c_int32), ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double),
                ("t_end_ms", C.c_double), ("device_ms", C.c_double), ("n", C.c_int32), ("m", C.c_int32),
                ("message", C.c_char * 160)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int32), ("completed", C.c_int32), ("pending", C.c_int32),
                ("active", C.c_int32), ("peak_active", C.c_int32), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


def register(L):
    vp = C.c_void_p
    L.vrprpd_alns_params_default.argtypes = [C.POINTER(AlnsParams)]
    L.vrprpd_alns_params_default.restype = None
    L.vrprpd_initial_solution.argtypes = [vp, C.POINTER(Solution)]
    L.vrprpd_initial_solution_paper.argtypes = [vp, C.c_int32, C.POINTER(Solution), vp]
    L.vrprpd_alns_run.argtypes = [vp, C.POINTER(Solution), C.POINTER(AlnsParams), C.c_uint64,
                                  C.POINTER(Solution), C.POINTER(Solution), C.POINTER(AlnsStats), vp, vp]
    L.vrprpd_insertion_matrix.argtypes = [vp, vp, vp, C.c_int32, vp, vp, vp]
    L.vrprpd_repair_then_matrix.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp,
                                            vp, vp, vp, vp]
    L.vrprpd_multi_create.argtypes = [vp, vp, vp, vp, C.c_int32, C.POINTER(vp)]
    L.vrprpd_multi_evaluate.argtypes = [vp, vp]
    L.vrprpd_multi_autotune.argtypes = [vp, vp, vp]
    L.vrprpd_multi_set_config.argtypes = [vp, vp]
    L.vrprpd_multi_destroy.argtypes = [vp]
    L.vrprpd_multi_destroy.restype = None
    L.vrprpd_brkga_params_default.argtypes = [C.POINTER(BrkgaParams)]
    L.vrprpd_brkga_params_default.restype = None
    L.vrprpd_brkga_decode.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp]
    L.vrprpd_brkga_run.argtypes = [vp, C.POINTER(BrkgaParams), C.POINTER(Solution), C.c_uint64,
                                   C.POINTER(Solution), vp, vp, vp, vp]
    L.vrprpd_server_create.argtypes = [C.c_size_t, C.c_int32, C.POINTER(vp)]
    L.vrprpd_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_int64)]
    L.vrprpd_server_poll.argtypes = [vp, C.c_int64, C.POINTER(Result), vp, vp]
    L.vrprpd_server_wait.argtypes = [vp, C.c_int64, C.POINTER(Result), vp, vp]
    L.vrprpd_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.vrprpd_server_cancel_pending.argtypes = [vp, vp]
    L.vrprpd_server_destroy.argtypes = [vp]
    L.vrprpd_server_destroy.restype = None
    return L
