"""ctypes declarations of the C ABI in ``include/nmf.h`` (same names).

Argument marshalling only: every step of the method runs in the CUDA
library.  Loading fails loudly if the library has not been built; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnmf_gb300.so")

NMF_OK, NMF_EINVAL, NMF_ENOMEM, NMF_ECUDA, NMF_ENOTCONV, NMF_ETIMEOUT, NMF_ECAPACITY, \
    NMF_ENUMERIC, NMF_ESTATE = range(9)
NMF_PREC_FP64, NMF_PREC_MIXED = 0, 1
NMF_DTYPE_F64, NMF_DTYPE_F32 = 0, 1
NMF_WARM_COLD, NMF_WARM_PREV, NMF_WARM_CHAIN = 0, 1, 2

# every symbol declared in include/nmf.h
EXPORTS = ("nmf_config_init", "nmf_create", "nmf_destroy", "nmf_append_columns", "nmf_num_columns",
           "nmf_set_factors", "nmf_get_factors", "nmf_sweep", "nmf_set_pass_mode",
           "nmf_objective_kkt", "nmf_status_string", "nmf_last_error", "nmf_launch_count",
           "nmf_set_timing", "nmf_get_timing", "nmf_get_pass_timing", "nmf_shard_buffer_len", "nmf_shard_y_half", "nmf_shard_x_half", "nmf_ipm", "nmf_ipm_direction", "nmf_save", "nmf_load", "nmf_get_config", "nmf_sweep_noalloc",
           "nmf_batch_create", "nmf_batch_destroy", "nmf_batch_size", "nmf_batch_problem",
           "nmf_batch_append_columns", "nmf_batch_set_factors", "nmf_batch_get_factors",
           "nmf_batch_set_pass_mode", "nmf_batch_set_schedule", "nmf_batch_sweep", "nmf_batch_autotune",
           "nmf_batch_launch_count", "nmf_batch_last_error", "nmf_selftest_bounded_wait", "nmf_selftest_tc16_wait", "nmf_measure_fma_peaks",
           "nmf_server_config_init", "nmf_server_create", "nmf_server_destroy", "nmf_server_open_stream",
           "nmf_server_submit", "nmf_server_close_stream", "nmf_server_poll", "nmf_server_get_factors",
           "nmf_server_get_stats", "nmf_server_last_error")

# exports whose return value is not an nmf_status
_NON_STATUS = ("nmf_config_init", "nmf_num_columns", "nmf_shard_buffer_len", "nmf_status_string", "nmf_last_error",
               "nmf_launch_count", "nmf_batch_size", "nmf_batch_problem", "nmf_batch_launch_count",
               "nmf_batch_last_error", "nmf_server_config_init", "nmf_server_last_error")


class nmf_config(C.Structure):
    _fields_ = [("n", C.c_int64), ("m_capacity", C.c_int64), ("k", C.c_int32), ("prec", C.c_int32),
                ("stol", C.c_double), ("kkt_target", C.c_double), ("mixed_switch", C.c_double),
                ("max_sweeps", C.c_int32), ("warm_start", C.c_int32), ("cuda_stream", C.c_void_p),
                ("kkt_abs_target", C.c_double)]


class nmf_stats(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("iter", C.c_int32), ("converged", C.c_int32),
                ("fp64_sweeps", C.c_int32), ("f", C.c_double), ("kkt_abs", C.c_double),
                ("kkt_rel", C.c_double), ("step_rel", C.c_double), ("changed_cols", C.c_int64),
                ("changed_rows", C.c_int64), ("nnls_notconv", C.c_int64), ("measured_iter", C.c_int32),
                ("entering_steps", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class nmf_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_streams", C.c_int32), ("max_sweeps_per_chunk", C.c_int32),
                ("sweeps_per_round", C.c_int32), ("pad", C.c_int32), ("kkt_target", C.c_double),
                ("mixed_switch", C.c_double), ("cuda_stream", C.c_void_p)]


class nmf_chunk_result(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("stream", C.c_int32), ("ncols", C.c_int32), ("t_submit_s", C.c_double),
                ("t_done_s", C.c_double), ("sweeps", C.c_int32), ("converged", C.c_int32),
                ("kkt_rel", C.c_double), ("f", C.c_double), ("m", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class nmf_server_stats(C.Structure):
    _fields_ = [("chunks_done", C.c_int64), ("columns_done", C.c_int64), ("rounds", C.c_int64),
                ("batch_sweeps", C.c_int64), ("stream_rounds", C.c_int64), ("max_streams_in_round", C.c_int32),
                ("streams_admitted", C.c_int32), ("streams_queued", C.c_int32), ("pad", C.c_int32),
                ("hbm_in_use_bytes", C.c_int64), ("hbm_budget_bytes", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class NMFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the built library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("the CUDA library %s has not been built; run "
                          "`python -m paper_2101_08431_gb300.build` (nvcc required)" % path)
    L = C.CDLL(path)
    H = C.c_void_p
    L.nmf_config_init.argtypes = [C.POINTER(nmf_config)]
    L.nmf_config_init.restype = None
    L.nmf_create.argtypes = [C.POINTER(nmf_config), C.POINTER(H)]
    L.nmf_destroy.argtypes = [H]
    L.nmf_append_columns.argtypes = [H, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32]
    L.nmf_num_columns.argtypes = [H]
    L.nmf_num_columns.restype = C.c_int64
    L.nmf_set_factors.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int32]
    L.nmf_get_factors.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    L.nmf_sweep.argtypes = [H, C.c_int32, C.POINTER(nmf_stats)]
    L.nmf_set_pass_mode.argtypes = [H, C.c_int32]
    L.nmf_objective_kkt.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
    L.nmf_status_string.argtypes = [C.c_int]
    L.nmf_status_string.restype = C.c_char_p
    L.nmf_last_error.argtypes = [H]
    L.nmf_last_error.restype = C.c_char_p
    L.nmf_launch_count.argtypes = [H]
    L.nmf_launch_count.restype = C.c_int64
    L.nmf_set_timing.argtypes = [H, C.c_int32]
    L.nmf_get_timing.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.nmf_get_pass_timing.argtypes = [H, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_int64)]
    L.nmf_shard_buffer_len.argtypes = [C.c_int64, C.c_int32]
    L.nmf_shard_buffer_len.restype = C.c_int64
    L.nmf_shard_y_half.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int32]
    L.nmf_shard_x_half.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(nmf_stats)]
    L.nmf_ipm.argtypes = [H, C.c_double, C.c_int32, C.POINTER(C.c_double)]
    L.nmf_ipm_direction.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    L.nmf_save.argtypes = [H, C.c_char_p]
    L.nmf_load.argtypes = [C.c_char_p, C.c_void_p, C.POINTER(H)]
    L.nmf_get_config.argtypes = [H, C.POINTER(nmf_config)]
    L.nmf_sweep_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    B = C.c_void_p
    L.nmf_batch_create.argtypes = [C.POINTER(nmf_config), C.c_int32, C.c_void_p, C.POINTER(B)]
    L.nmf_batch_destroy.argtypes = [B]
    L.nmf_batch_size.argtypes = [B]
    L.nmf_batch_size.restype = C.c_int32
    L.nmf_batch_problem.argtypes = [B, C.c_int32]
    L.nmf_batch_problem.restype = H
    L.nmf_batch_append_columns.argtypes = [B, C.c_int32, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                           C.c_int32]
    L.nmf_batch_set_factors.argtypes = [B, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]
    L.nmf_batch_get_factors.argtypes = [B, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int32]
    L.nmf_batch_set_pass_mode.argtypes = [B, C.c_int32]
    L.nmf_batch_set_schedule.argtypes = [B, C.c_int32, C.c_int32]
    L.nmf_batch_sweep.argtypes = [B, C.c_int32, C.POINTER(nmf_stats), C.POINTER(C.c_int32)]
    L.nmf_batch_autotune.argtypes = [B, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]
    L.nmf_batch_launch_count.argtypes = [B]
    L.nmf_batch_launch_count.restype = C.c_int64
    L.nmf_batch_last_error.argtypes = [B]
    L.nmf_batch_last_error.restype = C.c_char_p
    L.nmf_selftest_bounded_wait.argtypes = [C.c_int64, C.c_void_p]
    L.nmf_selftest_tc16_wait.argtypes = [C.c_int64, C.c_void_p]
    L.nmf_measure_fma_peaks.argtypes = [C.POINTER(C.c_double), C.c_void_p]
    S = C.c_void_p
    L.nmf_server_config_init.argtypes = [C.POINTER(nmf_server_config)]
    L.nmf_server_config_init.restype = None
    L.nmf_server_create.argtypes = [C.POINTER(nmf_server_config), C.POINTER(S)]
    L.nmf_server_destroy.argtypes = [S]
    L.nmf_server_open_stream.argtypes = [S, C.c_int64, C.c_int32, C.c_int64, C.c_uint64, C.POINTER(C.c_int32)]
    L.nmf_server_submit.argtypes = [S, C.c_int32, C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_uint64)]
    L.nmf_server_close_stream.argtypes = [S, C.c_int32]
    L.nmf_server_poll.argtypes = [S, C.POINTER(nmf_chunk_result), C.c_int32, C.POINTER(C.c_int32), C.c_int32]
    L.nmf_server_get_factors.argtypes = [S, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_int64)]
    L.nmf_server_get_stats.argtypes = [S, C.POINTER(nmf_server_stats)]
    L.nmf_server_last_error.argtypes = [S]
    L.nmf_server_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in _NON_STATUS:
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(status: int, handle=None, batch=None):
    if status != NMF_OK:
        L = load()
        detail = ""
        if handle:
            detail = L.nmf_last_error(handle).decode()
        elif batch:
            detail = L.nmf_batch_last_error(batch).decode()
        raise NMFError(status, "%s%s" % (L.nmf_status_string(status).decode(),
                                         (": " + detail) if detail else ""))
    return status
