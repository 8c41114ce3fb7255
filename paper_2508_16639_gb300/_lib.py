"""ctypes declarations of libescg's C ABI (include/escg.h).  Argument
marshalling only: every step of the Monte Carlo path runs in the CUDA
library.  Loading fails loudly if the library is missing -- there is no CPU
fallback."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libescg.so")

ESCG_OK, ESCG_EINVAL, ESCG_ENOMEM, ESCG_ECUDA, ESCG_ESTATE, ESCG_ETIMEOUT = 0, -1, -2, -3, -4, -5
STATUS_NAMES = {0: "ESCG_OK", -1: "ESCG_EINVAL", -2: "ESCG_ENOMEM", -3: "ESCG_ECUDA",
                -4: "ESCG_ESTATE", -5: "ESCG_ETIMEOUT"}


class Rates(C.Structure):
    _fields_ = [("interact", C.c_double), ("reproduce", C.c_double), ("exchange", C.c_double)]


class Options(C.Structure):
    _fields_ = [("p_empty", C.c_double), ("log_every", C.c_uint32),
                ("stop_at_extinction", C.c_int32), ("schedule_version", C.c_uint32),
                ("persistent", C.c_int32), ("cuda_stream", C.c_void_p),
                ("device_lattice", C.c_void_p), ("time_kernels", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("dominance_prob", C.POINTER(C.c_double)),
                ("neighbourhood", C.c_int32), ("reflecting_boundary", C.c_int32),
                ("height", C.c_int32), ("bits_per_site", C.c_int32), ("autotune", C.c_int32)]


class ReplicaSpec(C.Structure):
    _fields_ = [("L", C.c_int32), ("S", C.c_int32), ("digraph", C.POINTER(C.c_uint8)),
                ("rates", Rates), ("seed", C.c_uint64), ("p_empty", C.c_double),
                ("max_mcs", C.c_uint64), ("stop_at_extinction", C.c_int32),
                ("dominance_prob", C.POINTER(C.c_double))]


class BatchOptions(C.Structure):
    _fields_ = [("log_every", C.c_uint32), ("threads", C.c_int32), ("use_graph", C.c_int32),
                ("cuda_stream", C.c_void_p), ("resident", C.c_int32)]


class ServerOptions(C.Structure):
    _fields_ = [("arena_bytes", C.c_uint64), ("max_slots", C.c_int32), ("log_every", C.c_uint32),
                ("threads", C.c_int32), ("chunks_per_step", C.c_uint32), ("keep_lattice", C.c_int32),
                ("cuda_stream", C.c_void_p)]


_u8p = C.POINTER(C.c_uint8)
_u64p = C.POINTER(C.c_uint64)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)

# name -> (restype, argtypes); every symbol include/escg.h declares
SIGNATURES = {
    "escg_default_options": (None, [C.POINTER(Options)]),
    "escg_lattice_bytes": (C.c_size_t, [C.c_int32]),
    "escg_lattice_bytes_rect": (C.c_size_t, [C.c_int32, C.c_int32]),
    "escg_lattice_pitch_ex": (C.c_int32, [C.c_int32, C.c_int32]),
    "escg_lattice_bytes_ex": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "escg_lattice_pitch": (C.c_int32, [C.c_int32]),
    "escg_create": (C.c_void_p, [C.c_int32, C.c_int32, _u8p, C.POINTER(Rates), C.c_uint64]),
    "escg_create_ex": (C.c_void_p, [C.c_int32, C.c_int32, _u8p, C.POINTER(Rates), C.c_uint64,
                                    C.POINTER(Options)]),
    "escg_run": (C.c_int, [C.c_void_p, C.c_uint64]),
    "escg_sync": (C.c_int, [C.c_void_p]),
    "escg_counts": (C.c_int, [C.c_void_p, _u64p, _u64p]),
    "escg_counts_log": (C.c_int, [C.c_void_p, _u64p, _u64p, C.c_int64, _i64p]),
    "escg_snapshot": (C.c_int, [C.c_void_p, _u8p]),
    "escg_restore": (C.c_int, [C.c_void_p, _u8p, C.c_uint64]),
    "escg_step_host": (C.c_int, [C.c_void_p, _u8p, C.c_uint64, C.c_uint64, _u8p, _u64p]),
    "escg_step_host_async": (C.c_int, [C.c_void_p, _u8p, C.c_uint64, C.c_uint64, _u8p, _u64p]),
    "escg_step_host_wait": (C.c_int, [C.c_void_p]),
    "escg_device_lattice": (C.c_void_p, [C.c_void_p]),
    "escg_stream": (C.c_void_p, [C.c_void_p]),
    "escg_current_mcs": (C.c_uint64, [C.c_void_p]),
    "escg_launch_count": (C.c_uint64, [C.c_void_p]),
    "escg_destroy": (None, [C.c_void_p]),
    "escg_last_error": (C.c_char_p, []),
    "escg_exchange_from_mobility": (C.c_double, [C.c_double, C.c_int64]),
    "escg_circulant": (C.c_int, [C.c_int32, _i32p, C.c_int32, _u8p]),
    "escg_kernel_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), _u64p, C.c_int]),
    "escg_run_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _u8p, C.POINTER(Rates),
                                   C.c_uint64, C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "escg_batch_default_options": (None, [C.POINTER(BatchOptions)]),
    "escg_batch_create": (C.c_void_p, [C.c_int32, C.POINTER(ReplicaSpec), C.POINTER(BatchOptions)]),
    "escg_batch_run": (C.c_int, [C.c_void_p, C.c_uint64]),
    "escg_batch_sync": (C.c_int, [C.c_void_p]),
    "escg_batch_status": (C.c_int, [C.c_void_p, _u64p, _i32p, _u64p]),
    "escg_batch_active": (C.c_int32, [C.c_void_p]),
    "escg_batch_snapshot": (C.c_int, [C.c_void_p, C.c_int32, _u8p]),
    "escg_batch_threads": (C.c_int32, [C.c_void_p]),
    "escg_batch_uses_tma": (C.c_int32, [C.c_void_p]),
    "escg_batch_launch_count": (C.c_uint64, [C.c_void_p]),
    "escg_batch_destroy": (None, [C.c_void_p]),
    "escg_server_default_options": (None, [C.POINTER(ServerOptions)]),
    "escg_server_create": (C.c_void_p, [C.POINTER(ServerOptions)]),
    "escg_server_submit": (C.c_int64, [C.c_void_p, C.POINTER(ReplicaSpec)]),
    "escg_server_step": (C.c_int, [C.c_void_p, _i32p]),
    "escg_server_poll": (C.c_int, [C.c_void_p, _i64p, C.c_int32, _i32p]),
    "escg_server_result": (C.c_int, [C.c_void_p, C.c_int64, _u64p, _i32p, _u64p, _u8p]),
    "escg_server_stats": (C.c_int, [C.c_void_p, _i32p, _i32p, _u64p]),
    "escg_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "escg_server_threads": (C.c_int32, [C.c_void_p]),
    "escg_server_uses_tma": (C.c_int32, [C.c_void_p]),
    "escg_server_timing": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    "escg_server_launch_count": (C.c_uint64, [C.c_void_p]),
    "escg_server_destroy": (None, [C.c_void_p]),
    # include/escg_diag.h
    "escg_diag_int_throughput": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "escg_debug_stall_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint32]),
    "escg_coarse_blocks": (C.c_int32, [C.c_void_p]),
    "escg_update_kernel": (C.c_char_p, [C.c_void_p]),
    "escg_diag_alg_throughput": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "escg_autotune_result": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "escg_diag_l2_copy": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_double)]),
}

_lib = None


def load(path: str | None = None):
    """Loads libescg.so (built by paper_2508_16639_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libescg.so not found at {path}: run paper_2508_16639_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class EscgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int):
    if status != ESCG_OK:
        raise EscgError(status, load().escg_last_error().decode(errors="replace"))
