"""ctypes declarations of the C ABI in include/tpfa.h (argument marshalling only).

The shared library is built in-tree by ``paper_2304_11274_gb300.build``; if it
is missing, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpfa.so")

TPFA_OK = 0
ERRORS = {
    -1: "TPFA_ERR_INVALID_ARG",
    -2: "TPFA_ERR_OOM",
    -3: "TPFA_ERR_CUDA",
    -4: "TPFA_ERR_TOO_LARGE",
    -5: "TPFA_ERR_NONFINITE",
    -6: "TPFA_ERR_NO_STATE",
    -7: "TPFA_ERR_TIMEOUT",
    -8: "TPFA_ERR_DEVICE_CHECK",
    -9: "TPFA_ERR_NO_CONVERGENCE",
}
TPFA_FP64, TPFA_MIXED = 0, 1
KERNELS = {"auto": 0, "naive": 1, "tiled": 2, "tiled_tma": 3, "tiled2": 4}
PRECONDITIONERS = {"zline": 0, "jacobi": 1}


class TPFAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class TPFAParams(ctypes.Structure):
    _fields_ = [
        ("rho_ref", ctypes.c_double),
        ("p_ref", ctypes.c_double),
        ("c_f", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("g", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("c_r", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("dz", ctypes.c_double),
        ("connectivity", ctypes.c_int),
    ]


class TPFAKrylovOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("rtol", ctypes.c_double), ("check_every", ctypes.c_int),
                ("preconditioner", ctypes.c_int)]


class TPFAKrylovStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("breakdown", ctypes.c_int),
        ("b_norm", ctypes.c_double),
        ("rel_residual", ctypes.c_double),
    ]


# (name, restype, argtypes) of every exported symbol.
_VP, _I, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
SIGNATURES = [
    ("tpfa_create_grid", _I, [ctypes.POINTER(_VP), _I, _I, _I, ctypes.POINTER(TPFAParams), _I, _VP, _VP, _VP, _VP]),
    ("tpfa_set_state", _I, [_VP, _VP, _VP, _VP]),
    ("tpfa_set_pressure", _I, [_VP, _VP]),
    ("tpfa_assemble_residual", _I, [_VP, _VP, _VP]),
    ("tpfa_assemble_jacobian", _I, [_VP, _VP, _VP, _VP, _VP]),
    ("tpfa_assemble_jacobian_kernel", _I, [_VP, _I, _VP, _VP, _VP, _VP]),
    ("tpfa_resolve_kernel", _I, [_VP, _I, ctypes.POINTER(_I)]),
    ("tpfa_assemble_jacobian_host", _I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    ("tpfa_set_permeability", _I, [_VP, _VP, _VP]),
    ("tpfa_set_log_permeability", _I, [_VP, _VP, _VP]),
    ("tpfa_vjp", _I, [_VP, _VP, _VP, _VP, _VP]),
    ("tpfa_vjp_kernel", _I, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    ("tpfa_jvp", _I, [_VP, _VP, _VP, _VP, _VP]),
    ("tpfa_jvp_kernel", _I, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    ("tpfa_linear_solve", _I, [_VP, _VP, _VP, ctypes.POINTER(TPFAKrylovOpts), ctypes.POINTER(TPFAKrylovStats), _VP]),
    ("tpfa_newton_step", _I, [_VP, _VP, ctypes.POINTER(TPFAKrylovOpts), ctypes.POINTER(TPFAKrylovStats), _VP, _VP,
                              _VP]),
    ("tpfa_get_pattern", _I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_LL), _VP]),
    ("tpfa_copy_pattern", _I, [_VP, _VP, _VP, _VP]),
    ("tpfa_nnz", _LL, [_I, _I, _I, _I]),
    ("tpfa_grid_info", _I, [_VP] + [ctypes.POINTER(_I)] * 4 + [ctypes.POINTER(_LL), ctypes.POINTER(_I)]),
    ("tpfa_get_transmissibility", _I, [_VP, _I, _VP, _VP]),
    ("tpfa_sync_status", _I, [_VP, _VP]),
    ("tpfa_slab_bounds", _I, [_I, _I, _I] + [ctypes.POINTER(_I)] * 4),
    ("tpfa_create_slab", _I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _I, ctypes.POINTER(TPFAParams), _I, _VP, _VP, _VP,
                              _VP]),
    ("tpfa_slab_info", _I, [_VP] + [ctypes.POINTER(_I)] * 4 + [ctypes.POINTER(_LL)] * 4),
    ("tpfa_slab_exchange", _I, [_VP, _VP, _VP, _VP, _VP]),
    ("tpfa_set_tiling", _I, [_VP, _I, _I]),
    ("tpfa_get_tiling", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("tpfa_autotune", _I, [_VP, ctypes.c_char_p, _VP]),
    ("tpfa_create_mesh", _I, [ctypes.POINTER(_VP), _LL, _LL, ctypes.POINTER(TPFAParams), _I] + [_VP] * 7),
    ("tpfa_mesh_set_state", _I, [_VP, _VP, _VP, _VP]),
    ("tpfa_mesh_set_pressure", _I, [_VP, _VP]),
    ("tpfa_mesh_assemble", _I, [_VP, _VP, _VP, _VP, _VP]),
    ("tpfa_mesh_copy_pattern", _I, [_VP, _VP, _VP, _VP]),
    ("tpfa_mesh_info", _I, [_VP] + [ctypes.POINTER(_LL)] * 3 + [ctypes.POINTER(_I)]),
    ("tpfa_mesh_sync_status", _I, [_VP, _VP]),
    ("tpfa_destroy_mesh", _I, [_VP]),
    ("tpfa_create_ensemble", _I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP)]),
    ("tpfa_ensemble_set_outputs", _I, [_VP, _I, _VP, _VP, _VP]),
    ("tpfa_assemble_batch", _I, [_VP, _VP]),
    ("tpfa_ensemble_tiling", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_LL), ctypes.POINTER(_I)]),
    ("tpfa_ensemble_autotune", _I, [_VP, ctypes.c_char_p, _VP]),
    ("tpfa_destroy_ensemble", _I, [_VP]),
    ("tpfa_assemble_jacobian_static", _I, [_I, _I, _I, ctypes.POINTER(TPFAParams), _I] + [_VP] * 10),
    ("tpfa_static_workspace_bytes", _LL, [_I, _I, _I, _I, _I, _I]),
    ("tpfa_math_eval", _I, [_I, _VP, _VP, _LL, _VP]),
    ("tpfa_destroy", _I, [_VP]),
    ("tpfa_last_error_string", ctypes.c_char_p, []),
    ("tpfa_version", _I, []),
]

_lib = None


def load(path: str | None = None):
    """Load libtpfa.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build the CUDA library first "
            "(python -m paper_2304_11274_gb300.build, or __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(rc: int):
    if rc != TPFA_OK:
        msg = load().tpfa_last_error_string()
        raise TPFAError(rc, msg.decode() if msg else "")
    return rc
