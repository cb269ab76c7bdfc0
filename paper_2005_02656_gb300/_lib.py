"""ctypes binding of libsph (include/sph.h): structures, prototypes, loading.

Argument marshalling only; every computation runs in the library's CUDA
kernels.  Importing this module fails loudly if the library is not built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsph.so")

SPH_OK = 0
SPH_ERR_INVALID_ARG = -1
SPH_ERR_CUDA = -2
SPH_ERR_NB_OVERFLOW = -3
SPH_ERR_SINGULAR_IAD = -4
SPH_ERR_NONFINITE = -5
SPH_ERR_TIMEOUT = -6
SPH_ERR_OOM = -7
SPH_ERR_ORDER = -8

FLAG_NB_OVERFLOW = 0x1
FLAG_SINGULAR_IAD = 0x2
FLAG_NONFINITE = 0x4
FLAG_BAD_BOX = 0x8
FLAG_CELL_OVERFLOW = 0x10
FLAG_TIMEOUT = 0x20

SPH_FP64 = 0
SPH_FP32_MIXED = 1
SPH_KERNEL_EXACT = 0
SPH_KERNEL_TABLE = 1
SPH_PAIRS_STAGED = 0
SPH_PAIRS_LISTS = 1

STATE_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "h", "m", "u", "vxh", "vyh", "vzh", "du_prev",
                "rho", "p", "c", "iad", "ax", "ay", "az", "du", "omega")

# Every exported symbol of include/sph.h (checked by the ABI test).
EXPORTS = ("sph_default_params", "sph_init", "sph_destroy", "sph_set_params", "sph_kernel_norm",
           "sph_find_neighbors", "sph_get_neighbors", "sph_density", "sph_iad",
           "sph_momentum_energy", "sph_step", "sph_step_host", "sph_diagnostics",
           "sph_last_diagnostics", "sph_error_word", "sph_last_error", "sph_launch_count",
           "sph_profile", "sph_stage_times", "sph_stats", "sph_diagnostics_noalloc",
           "sph_ens_default_config", "sph_ensemble_init", "sph_ensemble_destroy",
           "sph_ensemble_set_config", "sph_ensemble_step", "sph_ensemble_capture",
           "sph_ensemble_replay", "sph_ensemble_error_word", "sph_ensemble_last_error",
           "sph_ensemble_info", "sph_ensemble_phase_times", "sph_gravity", "sph_adjoint_init", "sph_adjoint_destroy", "sph_adjoint_forward",
           "sph_adjoint_backward", "sph_adjoint_info", "sph_adjoint_time_steps",
           "sph_adjoint_last_error", "sph_measure_fp32_peak")
STAGES = ("sort", "find", "density", "iad", "momentum", "dt", "update")
ENS_PHASES = ("reset", "extent", "grid", "count", "scan", "items", "scatter", "order", "gather",
              "find", "density", "iad", "momentum", "dt", "update")


class SphState(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in STATE_FIELDS] + [("id", C.c_void_p), ("n", C.c_int64)]


class SphParams(C.Structure):
    _fields_ = [
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("periodic", C.c_int * 3),
        ("gamma", C.c_double), ("alpha", C.c_double), ("courant", C.c_double),
        ("dt_growth", C.c_double), ("ng_target", C.c_int), ("max_nb", C.c_int),
        ("sinc_n", C.c_double), ("precision", C.c_int), ("kernel_mode", C.c_int),
        ("gradh", C.c_int), ("pair_mode", C.c_int), ("energy_dt", C.c_double),
        ("angular_sums", C.c_int),
    ]


class EnsConfig(C.Structure):
    _fields_ = [("cell_factor", C.c_double), ("blocks_per_sm", C.c_int),
                ("test_skip_block", C.c_int), ("find_window", C.c_int),
                ("threads_per_particle", C.c_int), ("momentum_threads", C.c_int)]


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libsph error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libsph.so and declare its prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no fallback)")
    lib = C.CDLL(path)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    ctxp = C.c_void_p
    sp = C.POINTER(SphState)
    pp = C.POINTER(SphParams)
    lib.sph_default_params.argtypes = [pp]
    lib.sph_default_params.restype = None
    lib.sph_init.argtypes = [pp, I64, C.POINTER(ctxp)]
    lib.sph_init.restype = I
    lib.sph_destroy.argtypes = [ctxp]
    lib.sph_destroy.restype = None
    lib.sph_set_params.argtypes = [ctxp, pp]
    lib.sph_set_params.restype = I
    lib.sph_kernel_norm.argtypes = [ctxp]
    lib.sph_kernel_norm.restype = D
    for name in ("sph_find_neighbors", "sph_density", "sph_iad", "sph_momentum_energy"):
        f = getattr(lib, name)
        f.argtypes = [ctxp, sp, P]
        f.restype = I
    lib.sph_get_neighbors.argtypes = [ctxp, sp, P, P, P]
    lib.sph_get_neighbors.restype = I
    lib.sph_step.argtypes = [ctxp, sp, P, P]
    lib.sph_step.restype = I
    lib.sph_step_host.argtypes = [ctxp, sp, P, P]
    lib.sph_step_host.restype = I
    lib.sph_diagnostics.argtypes = [ctxp, sp, P, P]
    lib.sph_diagnostics.restype = I
    lib.sph_last_diagnostics.argtypes = [ctxp, P, P]
    lib.sph_last_diagnostics.restype = I
    lib.sph_error_word.argtypes = [ctxp, C.POINTER(C.c_uint32)]
    lib.sph_error_word.restype = I
    lib.sph_last_error.argtypes = [ctxp]
    lib.sph_last_error.restype = C.c_char_p
    lib.sph_launch_count.argtypes = [ctxp]
    lib.sph_launch_count.restype = I64
    ep = C.POINTER(EnsConfig)
    lib.sph_ens_default_config.argtypes = [ep]
    lib.sph_ens_default_config.restype = None
    lib.sph_ensemble_init.argtypes = [pp, I, P, P, P, P, P, C.POINTER(ctxp)]
    lib.sph_ensemble_init.restype = I
    lib.sph_ensemble_destroy.argtypes = [ctxp]
    lib.sph_ensemble_destroy.restype = None
    lib.sph_ensemble_set_config.argtypes = [ctxp, ep]
    lib.sph_ensemble_set_config.restype = I
    for name in ("sph_ensemble_step", "sph_ensemble_capture"):
        f = getattr(lib, name)
        f.argtypes = [ctxp, sp, P, I, P]
        f.restype = I
    lib.sph_ensemble_replay.argtypes = [ctxp, P]
    lib.sph_ensemble_replay.restype = I
    lib.sph_ensemble_error_word.argtypes = [ctxp, C.POINTER(C.c_uint32)]
    lib.sph_ensemble_error_word.restype = I
    lib.sph_ensemble_last_error.argtypes = [ctxp]
    lib.sph_ensemble_last_error.restype = C.c_char_p
    lib.sph_ensemble_info.argtypes = [ctxp, P]
    lib.sph_ensemble_info.restype = I
    lib.sph_ensemble_phase_times.argtypes = [ctxp, P, P]
    lib.sph_ensemble_phase_times.restype = I
    lib.sph_adjoint_init.argtypes = [pp, I64, I, I, C.POINTER(ctxp)]
    lib.sph_adjoint_init.restype = I
    lib.sph_adjoint_destroy.argtypes = [ctxp]
    lib.sph_adjoint_destroy.restype = None
    lib.sph_adjoint_forward.argtypes = [ctxp, sp, D, D, P, P]
    lib.sph_adjoint_forward.restype = I
    lib.sph_adjoint_backward.argtypes = [ctxp, P, P, P, P]
    lib.sph_adjoint_backward.restype = I
    lib.sph_adjoint_info.argtypes = [ctxp, P]
    lib.sph_adjoint_info.restype = I
    lib.sph_adjoint_time_steps.argtypes = [ctxp, P]
    lib.sph_adjoint_time_steps.restype = I
    lib.sph_adjoint_last_error.argtypes = [ctxp]
    lib.sph_adjoint_last_error.restype = C.c_char_p
    lib.sph_gravity.argtypes = [ctxp, sp, D, D, D, P, P, P, P, P]
    lib.sph_gravity.restype = I
    lib.sph_diagnostics_noalloc.argtypes = [sp, P, P]
    lib.sph_diagnostics_noalloc.restype = I
    lib.sph_stats.argtypes = [ctxp, P]
    lib.sph_stats.restype = I
    lib.sph_profile.argtypes = [ctxp, I]
    lib.sph_profile.restype = I
    lib.sph_stage_times.argtypes = [ctxp, P, P]
    lib.sph_stage_times.restype = I
    lib.sph_measure_fp32_peak.argtypes = [P, P]
    lib.sph_measure_fp32_peak.restype = I
    _lib = lib
    return lib


def check(lib, ctx, rc):
    if rc != SPH_OK:
        msg = lib.sph_last_error(ctx) if ctx else b""
        raise SphError(rc, (msg or b"").decode(errors="replace"))
    return rc
