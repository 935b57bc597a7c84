"""ctypes declarations of the C ABI in include/sps.h (argument marshalling only).

Loads the in-tree libsps.so and fails loudly when it is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsps.so")

SPS_OK = 0
STATUS_NAMES = {0: "SPS_OK", 1: "SPS_ERR_INVALID_ARG", 2: "SPS_ERR_CUDA", 3: "SPS_ERR_OOM",
                4: "SPS_ERR_DEGENERATE", 5: "SPS_ERR_NONFINITE", 6: "SPS_ERR_TIMEOUT",
                7: "SPS_ERR_STATE", 8: "SPS_ERR_UNSUPPORTED"}
MEM_HOST, MEM_DEVICE = 0, 1
PREC_SPLIT, PREC_FP32 = 0, 1
MKERNEL_RW, MKERNEL_MALA = 0, 1
PRIOR_ISO, PRIOR_DIAG, PRIOR_FULL = 0, 1, 2
RESAMPLE_MULTINOMIAL, RESAMPLE_RESIDUAL = 0, 1


class SpsPrior(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mean", C.POINTER(C.c_double)), ("cov_or_sd", C.POINTER(C.c_double))]


class SpsOptions(C.Structure):
    _fields_ = [("ess_fraction", C.c_double), ("h_init", C.c_double), ("h_step", C.c_double),
                ("h_min", C.c_double), ("h_max", C.c_double), ("target_accept", C.c_double),
                ("rne_cycle", C.c_double), ("rne_final", C.c_double), ("r_max", C.c_int32),
                ("precision", C.c_int32), ("mkernel", C.c_int32), ("cphase_block", C.c_int32),
                ("mala_target_accept", C.c_double), ("seed", C.c_uint64), ("resampling", C.c_int32),
                ("graphs", C.c_int32)]


class SpsSchedule(C.Structure):
    _fields_ = [("n_cycles", C.c_int32), ("cap_cycles", C.c_int32), ("t", C.POINTER(C.c_int64)),
                ("R", C.POINTER(C.c_int32)), ("cap_steps", C.c_int64), ("sigma", C.POINTER(C.c_double)),
                ("h", C.POINTER(C.c_double)), ("accept", C.POINTER(C.c_double))]


class SpsResult(C.Structure):
    _fields_ = [("mean", C.POINTER(C.c_double)), ("sd", C.POINTER(C.c_double)), ("nse", C.POINTER(C.c_double)),
                ("rne", C.POINTER(C.c_double)), ("log_ml_group", C.POINTER(C.c_double)),
                ("log_ml", C.c_double), ("log_ml_nse", C.c_double), ("log_ml_pooled", C.c_double),
                ("n_cycles", C.c_int32), ("m_steps", C.c_int64), ("seconds", C.c_double),
                ("log_pred", C.POINTER(C.c_double)), ("log_pred_nse", C.POINTER(C.c_double)),
                ("graph_steps", C.c_int64)]


class SpsTuneResult(C.Structure):
    _fields_ = [("tile_rows", C.c_int32), ("cluster", C.c_int32), ("chunk_obs", C.c_int32),
                ("n_candidates", C.c_int32), ("ms", C.c_double), ("ms_default", C.c_double)]


class SpsMstepInfo(C.Structure):
    _fields_ = [("h", C.c_double), ("accept_rate", C.c_double), ("rne_min", C.c_double), ("h_next", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)

# name -> (restype, argtypes); every symbol declared in include/sps.h
SIGNATURES = {
    "sps_options_default": (None, [C.POINTER(SpsOptions)]),
    "sps_init": (C.c_int, [C.POINTER(_P), _P, C.c_int64, C.c_int32, _P, C.c_int32, C.POINTER(SpsPrior),
                           C.POINTER(SpsOptions)]),
    "sps_destroy": (None, [_P]),
    "sps_set_stream": (C.c_int, [_P, _P]),
    "sps_status_string": (C.c_char_p, [C.c_int]),
    "sps_last_error": (C.c_char_p, [_P]),
    "sps_get_dims": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32)]),
    "sps_set_timing": (C.c_int, [_P, C.c_int32]),
    "sps_counters": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "sps_loglik": (C.c_int, [_P, _P, C.c_int64, C.c_int64, _P, C.c_int32, C.c_int32]),
    "sps_loglik_noalloc": (C.c_int, [_P, _P, C.c_int64, C.c_int64, _P]),
    "sps_loglik_grad": (C.c_int, [_P, _P, C.c_int64, C.c_int64, _P, _P, C.c_int32]),
    "sps_state_create": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(_P)]),
    "sps_state_destroy": (None, [_P]),
    "sps_state_get": (C.c_int, [_P, _P, _P, _P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "sps_state_result": (C.c_int, [_P, _P, C.POINTER(SpsResult)]),
    "sps_state_set": (C.c_int, [_P, _P, _P, _P, C.c_int64]),
    "sps_cphase": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_double), _P, _P]),
    "sps_sphase": (C.c_int, [_P, _P, _P, _P, C.c_int32]),
    "sps_mstep": (C.c_int, [_P, _P, C.c_int32, _P, _P, C.POINTER(SpsMstepInfo)]),
    "sps_mphase": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                             C.POINTER(C.c_double)]),
    "sps_run": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(SpsSchedule), C.POINTER(SpsSchedule),
                          C.POINTER(SpsResult)]),
    "sps_resample": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int32]),
    "sps_set_prior": (C.c_int, [_P, C.POINTER(SpsPrior)]),
    "sps_loglik_batched": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "sps_autotune": (C.c_int, [_P, C.c_int64, C.c_int64, C.POINTER(SpsTuneResult)]),
    "sps_run_batched": (C.c_int, [_P, C.c_int32, _P, C.c_double, C.c_int32, C.c_int32, C.POINTER(SpsResult)]),
    "sps_gprior": (C.c_int, [_P, C.c_double, _P, _P]),
    "sps_prior_normalize": (C.c_int, [C.c_int32, C.c_int32, _P, _P, _P, _P]),
    "sps_philox": (C.c_int, [_P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                             C.c_int64, _P, C.c_int32]),
    "sps_ess": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P, C.c_int32]),
    "sps_particle_cov": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int32]),
    "sps_rw_step_given": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int64, _P, _P, _P, C.c_int32, _P, _P, C.c_int32]),
    "sps_set_debug": (C.c_int, [_P, C.c_int32, C.c_uint64]),
    "sps_mala_step_given": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, C.c_int32]),
}

_lib = None


def load() -> C.CDLL:
    """Load libsps.so (built in-tree) and declare its signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_1304_4333_b300.build` "
                          "(the library has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SpsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
