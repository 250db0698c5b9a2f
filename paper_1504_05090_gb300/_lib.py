"""ctypes declarations of the libdqmc C ABI (include/dqmc.h).

Argument marshalling only: every step of the Monte Carlo path runs in the
CUDA library.  Importing this module raises if libdqmc.so has not been built;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdqmc.so")

DQMC_FP64 = 0
DQMC_FP32 = 1
DQMC_DF32 = 2
DQMC_GEMM_TENSOR = 0
DQMC_GEMM_FP64 = 1
DQMC_QR_BLOCKED = 0
DQMC_QR_PIVOTED = 1
MAX_SIDE = 16
MAX_DELAY = 32

ERRORS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "device out of memory",
          -4: "drift above limit", -5: "device-side wait timed out",
          -6: "non-finite or singular value", -7: "invalid state"}


class DqmcGroup(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
                ("t", ctypes.c_double), ("U", ctypes.c_double),
                ("beta", ctypes.c_double), ("dtau", ctypes.c_double),
                ("n_chains", ctypes.c_int32), ("stab_interval", ctypes.c_int32),
                ("delay_k", ctypes.c_int32), ("precision", ctypes.c_int32)]


class DqmcTiles(ctypes.Structure):
    _fields_ = [("kron_nv", ctypes.c_int32), ("wrap_nv", ctypes.c_int32),
                ("metro_ctas", ctypes.c_int32)]


# name -> (restype, argtypes); this list is also the export check of the tests.
SIGNATURES = {
    "dqmc_init": (ctypes.c_int, [ctypes.POINTER(DqmcGroup), ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "dqmc_init_at": (ctypes.c_int, [ctypes.POINTER(DqmcGroup), ctypes.c_int, ctypes.c_uint64,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "dqmc_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "dqmc_recompute_G": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_measure_Gtau": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "dqmc_measure_Gtau_origins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_int]),
    "dqmc_gtau_size": (ctypes.c_int64, [ctypes.c_void_p]),
    "dqmc_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int]),
    "dqmc_get_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_set_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_field_size": (ctypes.c_int64, [ctypes.c_void_p]),
    "dqmc_get_G": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "dqmc_get_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_reset_observables": (ctypes.c_int, [ctypes.c_void_p]),
    "dqmc_spin_correlation_size": (ctypes.c_int64, [ctypes.c_void_p]),
    "dqmc_get_spin_correlation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_correlation_length": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                               ctypes.c_int]),
    "dqmc_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "dqmc_num_chains": (ctypes.c_int, [ctypes.c_void_p]),
    "dqmc_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "dqmc_set_gemm_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "dqmc_set_qr_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "dqmc_set_metropolis_split": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "dqmc_use_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "dqmc_autotune": (ctypes.c_int, [ctypes.POINTER(DqmcGroup), ctypes.c_int, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(DqmcGroup)]),
    "dqmc_set_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(DqmcTiles)]),
    "dqmc_get_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(DqmcTiles)]),
    "dqmc_autotune_tiles": (ctypes.c_int, [ctypes.POINTER(DqmcGroup), ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.POINTER(DqmcTiles)]),
    "dqmc_timing_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "dqmc_timing_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int]),
    "dqmc_timing_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "dqmc_timing_class_name": (ctypes.c_char_p, [ctypes.c_int]),
    "dqmc_green_noalloc": (ctypes.c_int, [ctypes.POINTER(DqmcGroup), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "dqmc_trotter_extrapolate": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_int]),
    "dqmc_trotter_timing": (ctypes.c_int, [ctypes.c_void_p]),
    "dqmc_matsubara_sigma": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "dqmc_matsubara_timing": (ctypes.c_int, [ctypes.c_void_p]),
    "dqmc_destroy": (None, [ctypes.c_void_p]),
    "dqmc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "dqmc_last_cuda_error": (ctypes.c_char_p, [ctypes.POINTER(ctypes.c_int)]),
}


class DqmcError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, ERRORS.get(code, "unknown"), code))
        self.code = code


def load(path=LIB_PATH):
    """Load libdqmc.so and declare its entry points."""
    if not os.path.exists(path):
        raise ImportError("libdqmc.so is not built (%s); run paper_1504_05090_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def check(code, where, lib=None):
    if code < 0:
        err = DqmcError(code, where)
        if code == -2 and lib is not None:
            line = ctypes.c_int(0)
            msg = lib.dqmc_last_cuda_error(ctypes.byref(line)).decode()
            err = DqmcError(code, "%s [%s at libdqmc line %d]" % (where, msg, line.value))
        raise err
    return code
