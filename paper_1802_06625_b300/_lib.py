"""ctypes binding of libprune.so: the C ABI of include/prune.h, same names.

Argument marshalling only: every step of the dataflow runs in the CUDA
kernels of the library.  Importing this module loads the library and fails
loudly if it is missing (there is no CPU path).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P = ctypes.c_void_p
I32, I64, U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64

PRUNE_OK, PRUNE_EINVAL, PRUNE_ENOMEM, PRUNE_EAGAIN = 0, 1, 2, 3
PRUNE_ETIMEOUT, PRUNE_ECUDA, PRUNE_EBUSY, PRUNE_EDEVICE = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EAGAIN", 4: "ETIMEOUT", 5: "ECUDA",
                6: "EBUSY", 7: "EDEVICE"}
PRUNE_MEM_HOST, PRUNE_MEM_DEVICE, PRUNE_MEM_DEVICE_BORROW, PRUNE_MEM_DISCARD = 0, 1, 2, 3
PRUNE_RUN_ASYNC, PRUNE_RUN_SYNC, PRUNE_RUN_ACTORS, PRUNE_RUN_DEVICE_RULE, PRUNE_RUN_CUDA_CORES = 0, 1, 2, 4, 8
PRUNE_NUM_FIFOS = 8

EXPORTS = ("prune_fifo_capacity", "prune_graph_create", "prune_graph_destroy", "prune_push_frames",
           "prune_run", "prune_sync", "prune_pull", "prune_peek", "prune_fifo_stats",
           "prune_fifo_capacity_of", "prune_last_error", "prune_profile", "prune_kernel_times", "prune_fir_energy", "prune_det_sel", "prune_hx",
           "prune_fire_frames_noalloc", "prune_batch_create", "prune_batch_destroy", "prune_batch_offset",
           "prune_batch_fire", "prune_batch_sync", "prune_batch_pull", "prune_batch_last_error",
           "prune_hx_adjoint", "prune_fir_adjoint",
           "prune_batch_autotune", "prune_batch_set_tuning", "prune_batch_get_tuning",
           "prune_dpd_workspace_bytes", "prune_dpd_fire",
           "prune_model_create", "prune_model_destroy", "prune_model_add_actor", "prune_model_add_port",
           "prune_model_connect", "prune_model_set_control", "prune_model_check", "prune_model_dpg",
           "prune_model_dc", "prune_model_buffer_bound", "prune_model_classify", "prune_model_last_error",
           "prune_model_compile",
           "prune_server_create", "prune_server_destroy", "prune_server_open", "prune_server_submit",
           "prune_server_step", "prune_server_progress", "prune_server_poll", "prune_server_pull",
           "prune_server_close", "prune_server_sync", "prune_server_stats", "prune_server_last_error")
PRUNE_SERVER_AUTO_RELEASE = 1
PRUNE_BATCH_GRAPH = 1


class prune_graph_desc(ctypes.Structure):
    _fields_ = [("F", I32), ("B", I32), ("T", I32), ("N", I32), ("C", I32), ("out_frames", I32),
                ("tau", ctypes.c_float), ("taps", P), ("H", P), ("stream", P), ("device", I32),
                ("reserved", I32), ("hbm_budget", U64)]


class prune_frame_out(ctypes.Structure):
    _fields_ = [("frame", I64), ("c", I32), ("reserved", I32), ("idx", P), ("y", P)]


class prune_frame_view(ctypes.Structure):
    _fields_ = [("frame", I64), ("c", I32), ("reserved", I32), ("idx", P), ("y", P)]


class prune_batch_tuning(ctypes.Structure):
    _fields_ = [("fir_order", I32), ("hx_chunk", I32), ("hx_grid", I32), ("reserved", I32),
                ("ms", ctypes.c_double)]


class prune_model_report(ctypes.Structure):
    _fields_ = [("rate_errors", I32), ("type_errors", I32), ("rule_errors", I32 * 5), ("n_dpgs", I32),
                ("consistent", I32), ("first_error", ctypes.c_char * 256)]


class prune_compile_params(ctypes.Structure):
    _fields_ = [("B", I32), ("T", I32), ("N", I32), ("C", I32), ("tau", ctypes.c_float), ("out_frames", I32),
                ("taps", P), ("H", P), ("stream", P), ("device", I32), ("reserved", I32), ("hbm_budget", U64)]


class prune_compiled(ctypes.Structure):
    _fields_ = [("form", I32), ("units", I32), ("graph", prune_graph_desc), ("dpd_K", I32), ("dpd_T", I32),
                ("dpd_period", I64)]


class prune_server_desc(ctypes.Structure):
    _fields_ = [("B", I32), ("N", I32), ("F_max", I32), ("T_max", I32), ("max_streams", I32),
                ("frames_per_step", I32), ("ring", I32), ("max_inflight", I32), ("hbm_budget", U64),
                ("stream", P), ("device", I32), ("flags", I32)]


class PruneError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libprune.so not built at {path}: run `python -m paper_1802_06625_b300.build`")
    lib = ctypes.CDLL(path)
    sig = {
        "prune_fifo_capacity": [I64, I64, I64, ctypes.POINTER(I64)],
        "prune_graph_create": [ctypes.POINTER(prune_graph_desc), ctypes.POINTER(P)],
        "prune_graph_destroy": [P],
        "prune_push_frames": [P, P, I32, I32],
        "prune_run": [P, I32, ctypes.POINTER(I32), I32],
        "prune_sync": [P],
        "prune_pull": [P, P, I32, ctypes.POINTER(I32), I32],
        "prune_peek": [P, I32, ctypes.POINTER(prune_frame_view)],
        "prune_fifo_stats": [P, I32, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64)],
        "prune_fifo_capacity_of": [P, I32, ctypes.POINTER(I64)],
        "prune_profile": [P, I32],
        "prune_kernel_times": [P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), I32],
        "prune_fir_energy": [P, P, P, I32, I32, I32, I32, P, P, P, P],
        "prune_det_sel": [P, I32, I32, ctypes.c_float, P, P, P],
        "prune_hx": [P, P, P, I32, I32, I32, I32, P, P, P],
        "prune_fire_frames_noalloc": [P, P, P, P, I32, I32, I32, I32, I32, ctypes.c_float, P, P, P, P, P, P],
    }
    sig.update({
        "prune_batch_create": [ctypes.POINTER(prune_graph_desc), I32, ctypes.POINTER(P)],
        "prune_batch_destroy": [P],
        "prune_batch_offset": [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "prune_batch_fire": [P, P, I32],
        "prune_batch_sync": [P],
        "prune_batch_pull": [P, I32, ctypes.POINTER(prune_frame_out), I32],
        "prune_hx_adjoint": [P, P, P, I32, I32, I32, I32, P, P, P, P, P],
        "prune_batch_autotune": [P, P, I32, ctypes.POINTER(prune_batch_tuning), ctypes.POINTER(prune_batch_tuning),
                                 I32, ctypes.POINTER(I32)],
        "prune_batch_set_tuning": [P, ctypes.POINTER(prune_batch_tuning)],
        "prune_dpd_fire": [P, I64, I32, P, I32, I32, P, P, P, P, P, ctypes.c_size_t, P],
        "prune_model_create": [ctypes.POINTER(P)],
        "prune_model_destroy": [P],
        "prune_model_add_actor": [P, ctypes.c_char_p, I32, ctypes.POINTER(I32)],
        "prune_model_add_port": [P, I32, ctypes.c_char_p, I32, I32, I64, ctypes.POINTER(I32)],
        "prune_model_connect": [P, I32, I32, I64, I64, ctypes.POINTER(I32)],
        "prune_model_set_control": [P, I32, I32, I32],
        "prune_model_check": [P, ctypes.POINTER(prune_model_report)],
        "prune_model_dpg": [P, I32] + [ctypes.POINTER(I32)] * 6,
        "prune_model_dc": [P, I32, I32, ctypes.POINTER(I32), I32, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "prune_model_buffer_bound": [P, I32, ctypes.POINTER(I64)],
        "prune_model_classify": [P, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "prune_model_compile": [P, ctypes.POINTER(prune_compile_params), ctypes.POINTER(prune_compiled),
                                ctypes.POINTER(I32), ctypes.POINTER(I64), I32],
        "prune_batch_get_tuning": [P, ctypes.POINTER(prune_batch_tuning)],
        "prune_fir_adjoint": [P, P, P, I32, I32, I32, I32, P, P],
        "prune_server_create": [ctypes.POINTER(prune_server_desc), ctypes.POINTER(P)],
        "prune_server_destroy": [P],
        "prune_server_open": [P, ctypes.POINTER(prune_graph_desc), ctypes.POINTER(I64)],
        "prune_server_submit": [P, I64, P, I64, I64],
        "prune_server_step": [P, ctypes.POINTER(I32)],
        "prune_server_progress": [P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                  ctypes.POINTER(I64)],
        "prune_server_poll": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), I32, ctypes.POINTER(I32)],
        "prune_server_pull": [P, I64, ctypes.POINTER(prune_frame_out), I32],
        "prune_server_close": [P, I64],
        "prune_server_sync": [P],
        "prune_server_stats": [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(I32),
                               ctypes.POINTER(I64)],
    })
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.prune_last_error.argtypes = [P]
    lib.prune_last_error.restype = ctypes.c_char_p
    lib.prune_batch_last_error.argtypes = [P]
    lib.prune_batch_last_error.restype = ctypes.c_char_p
    lib.prune_dpd_workspace_bytes.argtypes = [I32, I32]
    lib.prune_dpd_workspace_bytes.restype = ctypes.c_size_t
    lib.prune_model_last_error.argtypes = [P]
    lib.prune_model_last_error.restype = ctypes.c_char_p
    lib.prune_server_last_error.argtypes = [P]
    lib.prune_server_last_error.restype = ctypes.c_char_p
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def check(status: int, g=None, batch=None, server=None, model=None):
    if status != PRUNE_OK:
        if model is not None:
            msg = lib().prune_model_last_error(model).decode(errors="replace")
        elif server is not None:
            msg = lib().prune_server_last_error(server).decode(errors="replace")
        elif batch is not None:
            msg = lib().prune_batch_last_error(batch).decode(errors="replace")
        else:
            msg = lib().prune_last_error(g).decode(errors="replace")
        raise PruneError(status, msg)
    return status
