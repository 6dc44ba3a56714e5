"""ctypes binding of liblbm.so (the C ABI of include/lbm.h and include/lbm_batch.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Loading fails loudly if the in-tree library has not been built; there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK = 0
LBM_ERR_INVALID = -1
LBM_ERR_SIZE = -2
LBM_ERR_CUDA = -3
LBM_ERR_NONFINITE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6
LBM_FP64 = 0
LBM_FP32_SHIFTED = 1
LBM_FP64_DF = 2
LBM_FLAG_PERIODIC_Y = 1
LBM_FLAG_REGULARIZED = 2
LBM_FLAG_TMA_LOADS = 4
LBM_FLAG_FP32_F64_TERMS = 8
LBM_FLAG_FP32_F64_COLLIDE = 16
LBM_PATH_PLAIN = 0
LBM_PATH_TMA = 1
LBM_NOALLOC_MAX_LX = 16384
LBM_NOBS = 8
LBM_BATCH_SHARED_TILES = 0
LBM_BATCH_PER_LATTICE = 1
LBM_BATCH_PARAM_TILES = 2

c_int = ctypes.c_int
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p
c_char_p = ctypes.c_char_p
P = ctypes.POINTER


class LbmParams(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("tau", c_double), ("g", c_double),
                ("t_top", c_double), ("t_bottom", c_double), ("rho0", c_double)]


class LbmLatticeDesc(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("tau", c_double), ("g", c_double),
                ("t_top", c_double), ("t_bottom", c_double), ("rho0", c_double),
                ("f_a", c_void_p), ("f_b", c_void_p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "lbm_state_bytes": (c_size_t, [P(LbmParams)]),
    "lbm_create": (c_int, [P(c_void_p), P(LbmParams), c_void_p, c_void_p, c_size_t, c_void_p]),
    "lbm_destroy": (None, [c_void_p]),
    "lbm_last_error": (c_char_p, [c_void_p]),
    "lbm_set_stream": (c_int, [c_void_p, c_void_p]),
    "lbm_init": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_step": (c_int, [c_void_p, c_int]),
    "lbm_step_from": (c_int, [c_void_p, c_void_p, c_void_p]),
    "lbm_step_graph": (c_int, [c_void_p, c_int]),
    "lbm_current": (c_void_p, [c_void_p]),
    "lbm_swap": (c_int, [c_void_p]),
    "lbm_step_columns": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int]),
    "lbm_pack_columns": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "lbm_unpack_columns": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "lbm_step_path": (c_int, [c_void_p]),
    "lbm_moments": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_profiles": (c_int, [c_void_p, c_void_p, c_void_p]),
    "lbm_step_observe": (c_int, [c_void_p, c_int, c_int, c_void_p, P(c_int)]),
    "lbm_get_state": (c_int, [c_void_p, c_void_p]),
    "lbm_set_state": (c_int, [c_void_p, c_void_p]),
    "lbm_propagate_bc": (c_int, [c_void_p, c_void_p, c_void_p]),
    "lbm_adjoint_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_adjoint_step_noalloc": (c_int, [P(LbmParams), c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_moments_vjp": (c_int, [c_void_p] * 7),
    "lbm_init_vjp": (c_int, [c_void_p] * 10),
    "lbm_adjoint_step_f32": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_moments_vjp_f32": (c_int, [c_void_p] * 7),
    "lbm_init_vjp_f32": (c_int, [c_void_p] * 10),
    "lbm_check_finite": (c_int, [c_void_p, c_void_p, P(c_int)]),
    "lbm_status": (c_int, [c_void_p]),
    "lbm_constants": (c_int, [c_void_p, P(c_double), P(c_double), P(c_double), P(c_double)]),
    "lbm_model_constants": (c_int, [P(LbmParams), P(c_double), P(c_double), P(c_double), P(c_double)]),
    "lbm_probe_fma": (c_int, [c_void_p, c_int, c_int, P(c_double), P(c_double)]),
    "lbm_probe_rcp": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_longlong]),
    "lbm_batch_tile_count": (c_int, []),
    "lbm_batch_tile_per_lattice": (c_int, [c_int]),
    "lbm_batch_tile_kind": (c_int, [c_int]),
    "lbm_batch_tile_shape": (c_int, [c_int, P(c_int), P(c_int)]),
    "lbm_batch_tile_rows": (c_int, [c_int]),
    "lbm_batch_create": (c_int, [P(c_void_p), c_int, P(LbmLatticeDesc), c_int, c_void_p]),
    "lbm_batch_destroy": (None, [c_void_p]),
    "lbm_batch_last_error": (c_char_p, [c_void_p]),
    "lbm_batch_init": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_batch_set_tile": (c_int, [c_void_p, c_int]),
    "lbm_batch_autotune": (c_int, [c_void_p, c_int, P(c_int), P(c_double)]),
    "lbm_batch_step": (c_int, [c_void_p, c_int]),
    "lbm_batch_step_persistent": (c_int, [c_void_p, c_int]),
    "lbm_batch_barrier_selftest": (c_int, [c_void_p, c_int]),
    "lbm_batch_current": (c_void_p, [c_void_p, c_int]),
    "lbm_batch_moments": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_batch_sites": (ctypes.c_longlong, [c_void_p]),
    "lbm_batch_status": (c_int, [c_void_p]),
}

_lib = None


def load():
    """Load the in-tree liblbm.so, or raise with instructions to build it."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1703_00186_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue  # symbol presence is checked by the tests against the headers
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code
