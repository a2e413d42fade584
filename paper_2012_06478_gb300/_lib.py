"""ctypes binding of librms.so (include/rms.h).  Argument marshalling only:
every step of the simulation runs in the library's CUDA kernels.  There is
no fallback: if the shared library is missing or fails to load, importing
this module raises."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librms.so")

RMS_OK = 0
RMS_W_PROB_RANGE = 1
RMS_W_LEAP_LIMIT = 2
RMS_E_INVALID_ARG = -1
RMS_E_OOM = -2
RMS_E_CUDA = -3
RMS_E_STEP_TOO_LARGE = -4
RMS_E_TIMEOUT = -6
RMS_E_CANCELLED = -7
RMS_E_BUSY = -8
RMS_E_DEVICE = -9
RMS_E_NOT_READY = -10
RMS_FP64 = 0
RMS_FP32 = 1
RMS_TRAJ_HASH = 1
RMS_CHECKED = 2
RMS_COUNTS = 4
RMS_MORTON = 8
RMS_EC = 0
RMS_RS = 1
RMS_ERL = 2
RMS_MAX_LEAPS = 64
RMS_PERM_KAPPA = 0
RMS_PERM_BAXTER = 1
RMS_SERVE_STEPS = 0
RMS_SERVE_FILL = 1
RMS_PEAK_FP64_ADD = 0
RMS_PEAK_FP64_MUL = 1
RMS_PEAK_FP64_FMA = 2
RMS_PEAK_GATHER = 3
RMS_PEAK_GATHER_DEP = 4


class RmsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rms status {status}: {msg}")
        self.status = status


class SubstrateDesc(C.Structure):
    _fields_ = [("labels", C.c_void_p), ("labels_on_device", C.c_int32),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("voxel_um", C.c_double), ("periodic", C.c_int32 * 3), ("n_labels", C.c_int32),
                ("D", C.c_void_p), ("T2", C.c_void_p), ("T1", C.c_void_p), ("kappa", C.c_void_p),
                ("kappa_scalar", C.c_double), ("rho", C.c_void_p), ("conc", C.c_void_p), ("lam", C.c_double),
                ("perm_model", C.c_int32), ("dead", C.c_void_p), ("stream", C.c_void_p)]


class SequenceDesc(C.Structure):
    _fields_ = [("dt_ms", C.c_double), ("n_steps", C.c_int64), ("n_shapes", C.c_int32), ("G", C.c_void_p),
                ("mode", C.c_void_p), ("n_dirs", C.c_int32), ("dirs", C.c_void_p), ("n_b", C.c_int32),
                ("b", C.c_void_p), ("n_rec", C.c_int32), ("rec_steps", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_int64), ("max_active", C.c_int32), ("steps_per_tick", C.c_int32),
                ("policy", C.c_int32)]


class RunDesc(C.Structure):
    _fields_ = [("n_walkers", C.c_int64), ("walker_begin", C.c_int64), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("flags", C.c_uint32), ("steps_per_launch", C.c_int32),
                ("interaction", C.c_int32), ("stream", C.c_void_p)]


class RunState(C.Structure):
    _fields_ = [("step", C.c_int64), ("i", C.c_void_p), ("o", C.c_void_p), ("i0", C.c_void_p), ("o0", C.c_void_p),
                ("c", C.c_void_p), ("A", C.c_void_p), ("phase", C.c_void_p), ("hash", C.c_void_p),
                ("moments", C.c_void_p)]


# name -> (argtypes, restype); the exported C entry points of include/rms.h
SIGNATURES = {
    "rms_version": ([], C.c_int),
    "rms_last_error": ([], C.c_char_p),
    "rms_create_substrate": ([C.POINTER(SubstrateDesc), C.POINTER(C.c_void_p)], C.c_int),
    "rms_destroy_substrate": ([C.c_void_p], C.c_int),
    "rms_set_sequence": ([C.c_void_p, C.POINTER(SequenceDesc), C.POINTER(C.c_void_p)], C.c_int),
    "rms_sequence_bvalues": ([C.c_void_p, C.c_void_p], C.c_int),
    "rms_destroy_sequence": ([C.c_void_p], C.c_int),
    "rms_run": ([C.c_void_p, C.POINTER(RunDesc), C.POINTER(C.c_void_p)], C.c_int),
    "rms_run_range": ([C.c_void_p, C.POINTER(RunDesc), C.POINTER(RunState), C.c_int64, C.POINTER(C.c_void_p)],
                      C.c_int),
    "rms_run_query": ([C.c_void_p], C.c_int),
    "rms_read_counts": ([C.c_void_p, C.c_void_p], C.c_int),
    "rms_read_slots": ([C.c_void_p, C.c_void_p], C.c_int),
    "rms_cancel": ([C.c_void_p], C.c_int),
    "rms_read_signal": ([C.c_void_p] + [C.c_void_p] * 4, C.c_int),
    "rms_read_walkers": ([C.c_void_p] + [C.c_void_p] * 8, C.c_int),
    "rms_read_partials": ([C.c_void_p] + [C.c_void_p] * 4, C.c_int),
    "rms_normalise_partials": ([C.c_int64, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "rms_philox4x32_10": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "rms_destroy_run": ([C.c_void_p], C.c_int),
    "rms_run_step_time_ms": ([C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "rms_server_create": ([C.POINTER(ServerConfig), C.POINTER(C.c_void_p)], C.c_int),
    "rms_server_submit": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_int32, C.POINTER(C.c_int64)],
                          C.c_int),
    "rms_server_poll": ([C.c_void_p, C.c_int64], C.c_int),
    "rms_server_wait": ([C.c_void_p, C.c_int64, C.c_int64] + [C.c_void_p] * 4, C.c_int),
    "rms_server_cancel": ([C.c_void_p, C.c_int64], C.c_int),
    "rms_server_request_info": ([C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "rms_server_stats": ([C.c_void_p, C.c_void_p], C.c_int),
    "rms_server_destroy": ([C.c_void_p], C.c_int),
    "rms_readout_noalloc": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                             C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    # include/rms_peaks.h
    "rms_measure_peak": ([C.c_int32, C.c_int64, C.c_double, C.c_int32, C.c_void_p, C.POINTER(C.c_double),
                          C.POINTER(C.c_double)], C.c_int),
    "rms_device_sm_count": ([C.POINTER(C.c_int32)], C.c_int),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2012_06478_gb300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def last_error() -> str:
    m = lib.rms_last_error()
    return m.decode() if m else ""


def check(status: int, allow=(RMS_OK,)) -> int:
    if status not in allow:
        raise RmsError(status, last_error())
    return status
