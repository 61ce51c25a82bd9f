"""ctypes declarations for libdamf.so (include/damf.h).  No fallback: the library must exist."""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# DAMF_LIB_VARIANT=check loads the build with device bounds checks (build.build(check=True))
LIB_PATH = os.path.join(HERE, "libdamf_check.so" if os.environ.get("DAMF_LIB_VARIANT") == "check" else "libdamf.so")

c_i32, c_i64, c_f64, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

STATUS_NAMES = {0: "DAMF_OK", 1: "DAMF_ERR_INVALID", 2: "DAMF_ERR_CAPACITY", 3: "DAMF_ERR_CUDA",
                4: "DAMF_ERR_NUMERIC", 5: "DAMF_ERR_TIMEOUT", 6: "DAMF_ERR_NOT_CONVERGED", 7: "DAMF_ERR_BOUNDS"}


class Config(ctypes.Structure):
    _fields_ = [("n", c_i32), ("n_capacity", c_i32), ("m_capacity", c_i64), ("d", c_i32), ("directed", c_i32),
                ("alpha", c_f64), ("eps", c_f64), ("refold_every", c_i32), ("rsvd_oversample", c_i32),
                ("rsvd_power_iters", c_i32), ("max_push_rounds", c_i32), ("precision", c_i32),
                ("threshold", c_i32)]


class Batch(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("op", ctypes.c_void_p),
                ("k", c_i32), ("new_nodes", c_i32), ("k_dev", ctypes.c_void_p)]


class State(ctypes.Structure):
    _fields_ = [("Ub", c_vp), ("Vb", c_vp), ("Zb", c_vp), ("r", c_vp), ("PU", c_vp), ("PV", c_vp), ("PUi", c_vp),
                ("PVi", c_vp), ("sigma", c_vp), ("s0", c_vp), ("updates_since_fold", c_i32)]


class Tuning(ctypes.Structure):
    _fields_ = [("push_blocks", c_i32), ("push_direct_chunks", c_i32)]


class Stats(ctypes.Structure):
    _fields_ = [("updates", c_i64), ("edges_applied", c_i64), ("entries_changed", c_i64), ("pushes", c_i64),
                ("push_edges", c_i64), ("push_rounds", c_i64), ("fixup_edges", c_i64), ("touched_rows", c_i64),
                ("folds", c_i64), ("last_rank", c_i32), ("last_status", c_i32), ("launches", c_i64),
                ("last_sweeps", c_i32), ("reserved", c_i32), ("jacobi_sweeps", c_i64), ("jacobi_full", c_i64),
                ("jacobi_gersh", c_i64),
                ("push_tasks", c_i64), ("push_items", c_i64), ("push_ns", c_i64 * 4)]


# every symbol include/damf.h declares, with its ctypes signature
SIGNATURES = {
    "damf_bytes_required": (c_sz, [ctypes.POINTER(Config)]),
    "damf_rsvd_width": (c_i32, [ctypes.POINTER(Config)]),
    "damf_init_factorize": (c_i32, [ctypes.POINTER(Config), c_vp, c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "damf_apply_edges": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_vp]),
    "damf_save_state": (c_i32, [c_vp, ctypes.POINTER(State), c_vp]),
    "damf_restore": (c_i32, [ctypes.POINTER(Config), c_vp, c_vp, c_i64, ctypes.POINTER(State), c_vp,
                             ctypes.POINTER(c_vp)]),
    "damf_apply_edges_host": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_vp]),
    "damf_apply_edges_counted": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_vp, c_i32, c_vp]),
    "damf_apply_edges_multi": (c_i32, [c_vp, c_i32, c_vp]),
    "damf_step_multi": (c_i32, [c_vp, c_i32, c_vp]),
    "damf_set_tuning": (c_i32, [c_vp, ctypes.POINTER(Tuning)]),
    "damf_fleet_create": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp)]),
    "damf_fleet_step": (c_i32, [c_vp, c_vp, c_vp]),
    "damf_fleet_set_shares": (c_i32, [c_vp, c_vp, c_f64]),
    "damf_fleet_set_weights": (c_i32, [c_vp, c_vp]),
    "damf_fleet_get_shares": (c_i32, [c_vp, c_vp, c_vp]),
    "damf_fleet_launches": (c_i64, [c_vp]),
    "damf_plan_slots": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp]),
    "damf_selftest_wait": (c_i32, [c_i32, c_i64, c_vp, c_vp]),
    "damf_debug_fail_allocations": (None, [c_i32]),
    "damf_fleet_set_timing": (c_i32, [c_vp, c_i32]),
    "damf_fleet_get_timing": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "damf_fleet_last_error": (ctypes.c_char_p, [c_vp]),
    "damf_fleet_destroy": (None, [c_vp]),
    "damf_get_tuning": (c_i32, [c_vp, ctypes.POINTER(Tuning)]),
    "damf_delete_nodes": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "damf_ppr_refresh": (c_i32, [c_vp, c_vp]),
    "damf_join": (c_i32, [c_vp, c_vp]),
    "damf_record_event": (c_i32, [c_vp, c_vp]),
    "damf_get_embeddings": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "damf_score_pairs": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_i32, c_vp, c_vp]),
    "damf_topk": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp]),
    "damf_num_nodes": (c_i32, [c_vp]),
    "damf_core_svd_workspace_size": (c_sz, [c_i32, c_i32]),
    "damf_core_svd": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "damf_core_svd_noalloc": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "damf_set_timing": (c_i32, [c_vp, c_i32]),
    "damf_get_timing": (c_i32, [c_vp, c_vp, c_vp]),
    "damf_get_state": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "damf_export_adjacency": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_i64]),
    "damf_get_last_touched": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "damf_get_stats": (c_i32, [c_vp, ctypes.POINTER(Stats)]),
    "damf_sync_status": (c_i32, [c_vp]),
    "damf_last_error": (ctypes.c_char_p, [c_vp]),
    "damf_destroy": (None, [c_vp]),
}

STAGES = ["prepare", "fixup", "gather", "chol", "core", "transforms", "scatter", "push", "fold"]

_lib = None


def load():
    """Loads libdamf.so; raises when it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdamf.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
