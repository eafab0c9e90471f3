"""Thin ctypes binding of include/x2c.h (argument marshalling only).

Every computation happens in libx2c_gb300.so; torch tensors only provide device memory
and streams.  The functions keep the C names (x2c_build_full, x2c_build_dlu, ...).
Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

X2C_OK = 0
STATUS_NAMES = {0: "X2C_OK", 1: "X2C_ERR_ARG", 2: "X2C_ERR_NOMEM", 3: "X2C_ERR_CUDA",
                4: "X2C_ERR_NOT_POSDEF", 5: "X2C_ERR_NOCONV", 6: "X2C_ERR_DECOUPLING",
                7: "X2C_ERR_NONFINITE", 8: "X2C_ERR_ADMISSION", 9: "X2C_ERR_TIMEOUT",
                10: "X2C_ERR_CANCELLED", 11: "X2C_ERR_NOT_FOUND"}
PREC_FP64, PREC_SPLIT_BF16 = 0, 1
DLU_FREE_ATOM, DLU_MOLECULAR_BLOCK = 0, 1
LOCAL_DLU, LOCAL_DLH = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)


class Options(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("two_component", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("dlu_potential", ctypes.c_int32),
                ("so_same_atom_only", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("local_approx", ctypes.c_int32), ("h_upper_only", ctypes.c_int32),
                ("decoupling", ctypes.c_int32)]


class Mats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("S", ctypes.c_void_p), ("T", ctypes.c_void_p),
                ("V", ctypes.c_void_p), ("W0", ctypes.c_void_p), ("Wx", ctypes.c_void_p),
                ("Wy", ctypes.c_void_p), ("Wz", ctypes.c_void_p)]


class HOut(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p * 4)]


class UOut(ctypes.Structure):
    _fields_ = [("UL", ctypes.c_void_p * 4), ("US", ctypes.c_void_p * 4)]


class Layout(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("atom_offset", ctypes.POINTER(ctypes.c_int32)),
                ("atom_kind", ctypes.POINTER(ctypes.c_int32)), ("n_kinds", ctypes.c_int32),
                ("kinds", ctypes.POINTER(Mats))]


class Counters(ctypes.Structure):
    _fields_ = [("pair_blocks", ctypes.c_int64), ("atomic_solves", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("credited_flops", ctypes.c_double)]


class SBasis(ctypes.Structure):
    _fields_ = [("n_nuc", ctypes.c_int32), ("n", ctypes.c_int32), ("nuc_xyz", ctypes.c_void_p),
                ("nuc_z", ctypes.c_void_p), ("bf_xyz", ctypes.c_void_p), ("bf_alpha", ctypes.c_void_p)]


class Property(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("LL", ctypes.c_void_p), ("SS", ctypes.c_void_p * 4)]


class GraphStats(ctypes.Structure):
    _fields_ = [("captures", ctypes.c_int64), ("replays", ctypes.c_int64), ("cached", ctypes.c_int32),
                ("last_replayed", ctypes.c_int32)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("reserved", ctypes.c_int32 * 4)]


class Request(ctypes.Structure):
    _fields_ = [("opt", Options), ("kind", ctypes.c_int32), ("memory", ctypes.c_int32), ("layout", Layout),
                ("kind_key", ctypes.POINTER(ctypes.c_uint64)), ("mol", Mats), ("ld", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("out", HOut), ("t_arrival", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("h", ctypes.c_void_p * 4),
                ("t_arrival", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("batch_size", ctypes.c_int32),
                ("cache_hits", ctypes.c_int32), ("cache_misses", ctypes.c_int32), ("slot", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "cancelled", "queued", "running",
                                              "builds_launched", "cache_hits", "cache_misses", "cache_entries",
                                              "cache_evictions")] + \
               [(k, ctypes.c_double) for k in ("latency_p50_ms", "latency_p99_ms", "latency_mean_ms",
                                               "latency_max_ms", "builds_per_s", "first_arrival",
                                               "last_completion")] + \
               [(k, ctypes.c_uint64) for k in ("bytes_in_use", "peak_bytes", "budget_bytes")] + \
               [("kernel_launches", ctypes.c_int64), ("max_concurrent", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "x2c_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "x2c_ctx_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "x2c_ctx_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "x2c_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "x2c_last_error_message": (ctypes.c_char_p, [ctypes.c_void_p]),
    "x2c_build_full": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Mats),
                                      ctypes.POINTER(HOut), ctypes.POINTER(UOut), ctypes.c_void_p]),
    "x2c_build_dlu": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Layout),
                                     ctypes.POINTER(Mats), ctypes.POINTER(HOut), ctypes.c_void_p]),
    "x2c_build_dlu_nab": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Layout),
                                         ctypes.POINTER(Mats), ctypes.c_void_p, ctypes.POINTER(HOut), ctypes.c_void_p]),
    "x2c_build_dlu_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Layout),
                                          ctypes.POINTER(Mats), ctypes.POINTER(HOut), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_void_p]),
    "x2c_dlu_partition": (ctypes.c_int, [ctypes.POINTER(Layout), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "x2c_build_dlu_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.c_int32,
                                             ctypes.POINTER(Layout), ctypes.POINTER(Mats),
                                             ctypes.POINTER(HOut), ctypes.c_void_p]),
    "x2c_atomic_transforms": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.c_int32,
                                             ctypes.POINTER(Mats), ctypes.POINTER(UOut), ctypes.c_void_p]),
    "x2c_atomic_transforms_noalloc": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.c_int32,
                                                     ctypes.POINTER(Mats), ctypes.POINTER(UOut), ctypes.c_void_p]),
    "x2c_build_dlu_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Layout),
                                          ctypes.POINTER(Mats), ctypes.POINTER(HOut), ctypes.c_void_p]),
    "x2c_quaternion_to_dense": (ctypes.c_int, [ctypes.c_void_p * 4, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "x2c_ctx_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Counters)]),
    "x2c_ctx_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "x2c_ctx_set_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "x2c_ctx_tuning_log": (ctypes.c_char_p, [ctypes.c_void_p]),
    "x2c_ctx_set_split_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "x2c_ctx_set_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "x2c_s_integrals": (ctypes.c_int, [ctypes.POINTER(SBasis), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "x2c_picture_change": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Layout),
                                          ctypes.POINTER(UOut), ctypes.POINTER(Property), ctypes.POINTER(HOut),
                                          ctypes.c_void_p]),
    "x2c_ctx_graph_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GraphStats)]),
    "x2c_query_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.c_int32,
                                           ctypes.POINTER(Layout), ctypes.POINTER(Mats),
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "x2c_ctx_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p,
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "x2c_build_dlu_with_transforms": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options), ctypes.POINTER(Layout),
                                                     ctypes.POINTER(UOut), ctypes.POINTER(Mats), ctypes.POINTER(HOut),
                                                     ctypes.c_void_p]),
    "x2c_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOptions), ctypes.POINTER(ctypes.c_void_p)]),
    "x2c_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "x2c_server_now": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "x2c_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "x2c_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "x2c_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(Result)]),
    "x2c_server_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "x2c_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "x2c_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "x2c_server_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
}


def exported_symbols():
    """Every function name declared in include/x2c.h that the binding exposes."""
    return sorted(_SIGS)


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libx2c_gb300.so (building it first if asked); raise if it is unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB_PATH
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build_library()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class X2CError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} {detail}".strip())


def check(code, where, ctx=None):
    if code != X2C_OK:
        detail = ""
        if ctx is not None and code == 3:
            detail = load().x2c_last_error_message(ctx).decode()
        raise X2CError(code, where, detail)
