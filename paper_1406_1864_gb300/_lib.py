"""ctypes view of the C ABI in include/fwi.h (argument marshalling only).

Loads the in-tree libfwi.so. If it is missing or older than its sources it is
built with nvcc first; if that is impossible the import fails loudly: there is
no CPU fallback of any step of the path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_float, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                                ctypes.c_void_p, ctypes.c_size_t)

FWI_OK, FWI_ERR_INVALID_ARG, FWI_ERR_CFL, FWI_ERR_NOMEM, FWI_ERR_CUDA, FWI_ERR_TIMEOUT, \
    FWI_ERR_UNSTABLE = range(7)
STATUS_NAMES = ["FWI_OK", "FWI_ERR_INVALID_ARG", "FWI_ERR_CFL", "FWI_ERR_NOMEM", "FWI_ERR_CUDA",
                "FWI_ERR_TIMEOUT", "FWI_ERR_UNSTABLE"]
FWI_MISFIT_OLS, FWI_MISFIT_TIME_INTEGRAL = 0, 1
FWI_ILLUM_U2, FWI_ILLUM_UTT2 = 0, 1
FWI_PRECOND_NONE, FWI_PRECOND_ILLUM, FWI_PRECOND_OFFSET = 0, 1, 2
FWI_CKPT_SPONGE, FWI_CKPT_SNAPSHOT = 0, 1
FWI_SNAP_F32, FWI_SNAP_BF16, FWI_SNAP_F16S = 0, 1, 2
(FWI_OP_FORWARD, FWI_OP_FORWARD_SAVE, FWI_OP_GRADIENT, FWI_OP_ILLUMINATION,
 FWI_OP_OFFSET_HESSIAN, FWI_OP_PRECONDITION, FWI_OP_BORN, FWI_OP_GN_HVP, FWI_OP_MISFIT,
 FWI_OP_RECEIVER_FACTOR, FWI_OP_PRECONDITION_RECEIVER, FWI_OP_EXT_BORN, FWI_OP_EXT_MIGRATION,
 FWI_OP_PM_HESSIAN) = range(14)
FWI_HEXT_LIMIT = 6
FWI_RECV_PLESSIX_MULDER, FWI_RECV_GREEN = 0, 1
FWI_CFL_LIMIT_2D, FWI_CFL_LIMIT_3D = 0.5546, 0.4528  # v dt / dx limits (include/fwi.h)
FWI_HMAX_LIMIT = 12
FWI_BATCH_MAX = 4


class FwiGrid(ctypes.Structure):
    _fields_ = [("ndim", c_int), ("nz", c_int), ("ny", c_int), ("nx", c_int), ("dx", c_float),
                ("dt", c_float), ("nt", c_int), ("sponge", c_int), ("vref", c_float),
                ("refl", c_float)]


class FwiGeometry(ctypes.Structure):
    _fields_ = [("nshots", c_int), ("nrec", c_int), ("src", c_void_p), ("rec", c_void_p),
                ("wavelet", c_void_p)]


class FwiOptions(ctypes.Structure):
    _fields_ = [("misfit", c_int), ("illum_mode", c_int), ("hmax", c_int), ("precond", c_int),
                ("eps", c_float), ("ckpt", c_int), ("snap_prec", c_int), ("snap_interval", c_int),
                ("shot_group", c_int), ("hess_v6", c_int)]


class FwiPhaseTimes(ctypes.Structure):
    _fields_ = [("forward_ms", c_float), ("adjoint_ms", c_float), ("other_ms", c_float),
                ("forward_launches", c_int), ("adjoint_launches", c_int),
                ("other_launches", c_int)]


P = ctypes.POINTER
_SIGS = {
    "fwi_workspace_bytes": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_int, P(c_size_t)],
    "fwi_forward": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_int, c_void_p,
                    c_size_t, c_void_p],
    "fwi_adjoint_apply": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_void_p,
                          c_void_p, c_size_t, c_void_p],
    "fwi_adjoint_gradient": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                             c_void_p],
    "fwi_illumination": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_void_p,
                         c_size_t, c_void_p],
    "fwi_offset_hessian_diag": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p,
                                c_void_p, c_size_t, c_void_p],
    "fwi_misfit": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_void_p, c_void_p,
                   c_size_t, c_void_p],
    "fwi_receiver_factor": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_int, c_void_p, c_void_p, c_void_p,
                            c_size_t, c_void_p],
    "fwi_plessix_mulder_hessian": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_void_p,
                                   c_size_t, c_void_p],
    "fwi_precondition_receiver": [P(FwiGrid), c_void_p, c_void_p, c_int, c_int, c_void_p, c_int, c_float,
                                  c_void_p, c_void_p, c_size_t, c_void_p],
    "fwi_extended_born": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_int, c_void_p, c_void_p, c_void_p,
                          c_void_p, c_size_t, c_void_p],
    "fwi_extended_migration": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_int, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_size_t, c_void_p],
    "fwi_selftest_wait": [ctypes.c_uint, c_void_p, c_size_t, c_void_p],
    "fwi_born": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_void_p, c_void_p,
                 c_size_t, c_void_p],
    "fwi_gauss_newton_hvp": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_void_p,
                             c_void_p, c_size_t, c_void_p],
    "fwi_precondition": [P(FwiGrid), c_void_p, c_void_p, c_int, c_int, c_float, c_void_p, c_void_p,
                         c_size_t, c_void_p],
    "fwi_forward_noalloc": [P(FwiGrid), P(FwiGeometry), c_void_p, c_void_p, c_void_p],
    "fwi_batch_workspace_bytes": [c_int, P(FwiGrid), P(FwiGeometry), P(FwiOptions), P(c_size_t)],
    "fwi_batch_gradient": [c_int, P(FwiGrid), P(FwiGeometry), P(FwiOptions), P(c_void_p), P(c_void_p),
                           P(c_void_p), P(c_void_p), c_void_p, P(c_void_p), P(c_void_p), c_void_p,
                           c_size_t, c_void_p],
    "fwi_exec_gradient_create": [c_int, P(FwiGrid), P(FwiGeometry), P(FwiOptions), P(c_void_p),
                                 P(c_void_p), P(c_void_p), P(c_void_p), c_void_p, P(c_void_p),
                                 P(c_void_p), c_void_p, c_size_t, c_void_p, P(c_void_p)],
    "fwi_exec_run": [c_void_p, c_void_p],
    "fwi_exec_input_ready": [c_void_p, c_void_p],
    "fwi_autotune": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), c_void_p, c_void_p, c_size_t, c_void_p,
                     P(c_int)],
    "fwi_autotune_reset": [],
    "fwi_autotune_set": [P(FwiGrid), P(FwiGeometry), P(FwiOptions), P(c_int)],
    "fwi_exec_destroy": [c_void_p],
    "fwi_profile_enable": [c_int],
    "fwi_profile_last": [P(FwiPhaseTimes)],
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """The loaded libfwi.so (built first if stale and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        try:
            _build.build()
        except (OSError, FileNotFoundError) as e:  # no nvcc on this machine
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libfwi.so is not built and cannot be built here: {e}") from e
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libfwi.so is not built: run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = c_int
    lib.fwi_last_error.argtypes = []
    lib.fwi_last_error.restype = ctypes.c_char_p
    lib.fwi_version.argtypes = []
    lib.fwi_version.restype = c_int
    _lib = lib
    return lib


class FwiError(RuntimeError):
    """A non-OK status from the library, with its message."""

    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{func}: {name}: {msg}")


def check(status: int, func: str):
    if status != FWI_OK:
        raise FwiError(status, func, load().fwi_last_error().decode(errors="replace"))
