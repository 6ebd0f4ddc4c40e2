"""ctypes binding of libtrg (include/trg.h): argument marshalling only.

Every computation happens in the CUDA library; this module loads it (building
it in-tree first if it is missing or older than its sources) and fails loudly
if it cannot.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int, c_double, c_size_t, c_void_p, c_uint64 = (ctypes.c_int, ctypes.c_double, ctypes.c_size_t,
                                                  ctypes.c_void_p, ctypes.c_uint64)
P_double = ctypes.POINTER(ctypes.c_double)
P_int = ctypes.POINTER(ctypes.c_int)

TRG_OK, TRG_EINVAL, TRG_ESTATE, TRG_ENOMEM, TRG_ENUMERIC, TRG_ETIMEOUT, TRG_ECUDA, TRG_ENOTSUP = range(8)
TRG_ISING, TRG_XY, TRG_POTTS = 0, 1, 2
TRG_FP64, TRG_SPLIT_BF16 = 0, 1
TRG_TRUNC_PAPER, TRG_TRUNC_MULTIPLET = 0, 1

# Every exported symbol of include/trg.h with (restype, argtypes).
ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class trg_config(ctypes.Structure):
    _fields_ = [
        ("precision", c_int),
        ("split_slices", c_int),
        ("split_from_step", c_int),
        ("trunc", c_int),
        ("gap_tol", c_double),
        ("oversample", c_int),
        ("eig_tol", c_double),
        ("eig_max_iter", c_int),
        ("seed", c_uint64),
        ("workspace_bytes", c_size_t),
        ("mma_pairs", c_int),
        ("fused_slices", c_int),
        ("fp64_max_dd", c_int),
        ("env_slices", c_int),
        ("autotune", c_int),
    ]


class trg_phase_stats(ctypes.Structure):
    _fields_ = [("ms", c_double), ("calls", c_uint64), ("flops", c_double), ("mma_flops", c_double)]


PHASES = ("env", "eig", "x1", "x2", "x3", "norm", "mma", "mma_x2")
TRG_EAGAIN, TRG_ECANCELED = 8, 9
TRG_SERVE_FIFO, TRG_SERVE_SHORTEST_FIRST = 0, 1
TRG_DRY_RUN_FAIL_SEED = 0xFA17FA17


class trg_solve_spec(ctypes.Structure):
    _fields_ = [("model", c_int), ("beta", c_double), ("h", c_double), ("D0", c_int), ("Dcut", c_int),
                ("nsteps", c_int), ("precision", c_int), ("split_slices", c_int), ("trunc", c_int),
                ("seed", c_uint64)]


class trg_solve_result(ctypes.Structure):
    _fields_ = [("status", c_int), ("f", c_double), ("lnz_per_site", c_double), ("seconds_queued", c_double),
                ("seconds_run", c_double), ("slot", c_int)]


class trg_server_config(ctypes.Structure):
    _fields_ = [("slots", c_int), ("hbm_budget_bytes", c_size_t), ("workspace_bytes", c_size_t),
                ("dry_run", c_int), ("dry_run_seconds_per_step", c_double), ("policy", c_int),
                ("max_wait_s", c_double)]


class trg_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("failed", c_uint64), ("cancelled", c_uint64),
                ("running", c_uint64), ("queued", c_uint64), ("bytes_in_use", c_size_t), ("peak_bytes", c_size_t),
                ("p50_latency_s", c_double), ("p99_latency_s", c_double), ("max_latency_s", c_double),
                ("solves_per_s", c_double)]

SIGNATURES = {
    "trg_config_default": (c_int, [ctypes.POINTER(trg_config)]),
    "trg_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(trg_config)]),
    "trg_destroy": (c_int, [c_void_p]),
    "trg_set_stream": (c_int, [c_void_p, c_void_p]),
    "trg_set_allocator": (c_int, [c_void_p, ALLOC_FN, FREE_FN, c_void_p]),
    "trg_set_precision": (c_int, [c_void_p, c_int, c_int, c_int]),
    "trg_set_wait_limit": (c_int, [c_void_p, c_uint64]),
    "trg_init_tensor": (c_int, [c_void_p, c_int, c_double, c_double, c_int]),
    "trg_init_tensor_raw": (c_int, [c_void_p, P_double, c_int, c_int, c_double]),
    "trg_init_impure": (c_int, [c_void_p]),
    "trg_init_impure_raw": (c_int, [c_void_p, P_double]),
    "trg_expectation": (c_int, [c_void_p, P_double]),
    "trg_coarse_grain": (c_int, [c_void_p, c_int, c_int]),
    "trg_free_energy": (c_int, [c_void_p, P_double, P_double]),
    "trg_shard_extent": (c_int, [c_void_p, P_int]),
    "trg_shard_begin": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_size_t, P_int]),
    "trg_shard_finish": (c_int, [c_void_p, c_void_p, c_int]),
    "trg_solve3d": (c_int, [c_void_p, c_int, c_double, c_double, c_int, c_int, P_double, P_double]),
    "trg_get_spectrum": (c_int, [c_void_p, c_int, P_double, c_int, P_int]),
    "trg_get_state": (c_int, [c_void_p, P_int, P_int, P_int, P_double]),
    "trg_get_tensor": (c_int, [c_void_p, P_double, c_size_t]),
    "trg_environment": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "trg_isometry": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, P_double, P_int]),
    "trg_contract": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "trg_gemm": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int]),
    "trg_gemm_noalloc": (c_int, [c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_int,
                                 c_void_p]),
    "trg_profile_enable": (c_int, [c_void_p, c_int]),
    "trg_profile_read": (c_int, [c_void_p, c_int, ctypes.POINTER(trg_phase_stats)]),
    "trg_server_config_default": (c_int, [ctypes.POINTER(trg_server_config)]),
    "trg_solve_spec_default": (c_int, [ctypes.POINTER(trg_solve_spec)]),
    "trg_solve_bytes": (c_size_t, [ctypes.POINTER(trg_solve_spec), c_size_t]),
    "trg_serve_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(trg_server_config)]),
    "trg_serve_submit": (c_int, [c_void_p, ctypes.POINTER(trg_solve_spec), ctypes.POINTER(c_uint64)]),
    "trg_serve_poll": (c_int, [c_void_p, c_uint64, ctypes.POINTER(trg_solve_result)]),
    "trg_serve_wait": (c_int, [c_void_p, c_uint64, c_double, ctypes.POINTER(trg_solve_result)]),
    "trg_serve_cancel": (c_int, [c_void_p, c_uint64]),
    "trg_serve_get_stats": (c_int, [c_void_p, ctypes.POINTER(trg_serve_stats)]),
    "trg_serve_destroy": (c_int, [c_void_p]),
    "trg_batch_run": (c_int, [c_int, ctypes.POINTER(trg_solve_spec), c_int, ctypes.POINTER(trg_server_config),
                              ctypes.POINTER(trg_solve_result)]),
    "trg_status_string": (ctypes.c_char_p, [c_int]),
    "trg_last_error": (ctypes.c_char_p, [c_void_p]),
    "trg_launch_count": (c_uint64, [c_void_p]),
    "trg_get_counters": (c_int, [c_void_p, ctypes.POINTER(c_uint64), c_int]),
}

_lock = threading.Lock()
_lib = None


class TRGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libtrg, compiling it in-tree first if needed.  Raises if the
    library cannot be built or loaded: the product path has no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_needed and _build.stale():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libtrg is not built ({path}); run __graft_entry__.build()")
        so = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(so, name)
            fn.restype = res
            fn.argtypes = args
        _lib = so
        return so


def check(status: int, ctx=None, what: str = ""):
    if status == TRG_OK:
        return
    lib = load()
    msg = lib.trg_status_string(status).decode()
    if ctx:
        detail = lib.trg_last_error(ctx).decode()
        if detail:
            msg = f"{msg}: {detail}"
    raise TRGError(status, f"{what}: {msg}" if what else msg)
