"""ctypes binding of libslab.so (argument marshalling only; every step runs in the CUDA library)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int, c_double, c_void_p, c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64

SLAB_OK, SLAB_EINVAL, SLAB_ENOMEM, SLAB_ESINGULAR, SLAB_ENOCONV, SLAB_ETIMEOUT, SLAB_ECUDA, SLAB_EUNSUPPORTED = range(8)
POISSON, DIFFUSION, HELMHOLTZ, CONVECTION = 0, 1, 2, 3
KERNEL_CLASSES = ("coeff", "tree_factor", "assemble_T", "panel", "trailing", "schur_update", "sweep_products",
                  "tree_up", "tree_down", "stencil", "other", "slab_panel", "slab_trailing", "slab_schur")
PREC_FP64, PREC_FP32, PREC_TF32, PREC_FP64_TC = 0, 1, 2, 3


class SlabGrid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int)]


class SlabCoeffs(ctypes.Structure):
    _fields_ = [("kind", c_int), ("kappa", c_void_p), ("c", c_void_p), ("omega", c_double), ("beta", c_void_p)]


class SlabOpts(ctypes.Structure):
    _fields_ = [("factor_prec", c_int), ("pivot", c_int), ("rtol", c_double), ("max_refine", c_int),
                ("krylov", c_int), ("stream", c_void_p), ("profile", c_int),
                ("stage2", c_int), ("interface_prec", c_int)]


class SlabError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _strerror(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


_LIB = None
_LOCK = threading.Lock()

# name -> (restype, argtypes): every function declared in include/slab.h
SIGNATURES = {
    "slab_default_opts": (None, [ctypes.POINTER(SlabOpts)]),
    "slab_factor": (c_int, [ctypes.POINTER(SlabGrid), ctypes.POINTER(SlabCoeffs), c_int,
                            ctypes.POINTER(SlabOpts), ctypes.POINTER(c_void_p)]),
    "slab_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.POINTER(c_double),
                           ctypes.POINTER(c_int)]),
    "slab_apply_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "slab_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "slab_apply_transpose": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "slab_boundary_lift": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "slab_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "slab_reduced_rhs": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "slab_interface_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "slab_interior_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "slab_get_T_block": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "slab_apply_T": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "slab_sizes": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64), ctypes.POINTER(c_int)]),
    "slab_device_bytes": (c_int64, [c_void_p]),
    "slab_stage2_order": (c_int, [c_void_p]),
    "slab_last_error": (c_int, [c_void_p]),
    "slab_destroy": (None, [c_void_p]),
    "slab_strerror": (ctypes.c_char_p, [c_int]),
    "slab_profile": (c_int, [c_void_p, c_int]),
    "slab_profile_read": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "slab_tc_gemm": (c_int, [c_int, c_int, c_int, ctypes.c_float, c_void_p, c_int64, c_void_p, c_int64,
                             ctypes.c_float, c_void_p, c_int64, c_int, c_int, c_void_p, c_void_p]),
    "slab_residual_norms_noalloc": (c_int, [c_int, c_int, c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                                            c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "slab_fp64_tc_gemm": (c_int, [c_int, c_int, c_int, c_double, c_void_p, c_int64, c_void_p, c_int64, c_void_p,
                                  c_int64, c_void_p, c_void_p, c_void_p]),
    "slab_fp64_tc_gemm_work_bytes": (ctypes.c_size_t, [c_int, c_int, c_int]),
    "slab_batch_create": (c_int, [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(SlabOpts),
                                  c_int, c_int, c_int, ctypes.POINTER(c_void_p)]),
    "slab_batch_buffers": (c_int, [c_void_p, c_int] + [ctypes.POINTER(c_void_p)] * 6),
    "slab_batch_run": (c_int, [c_void_p, c_void_p]),
    "slab_batch_results": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "slab_batch_device_bytes": (c_int64, [c_void_p]),
    "slab_batch_destroy": (None, [c_void_p]),
    "slab_autotune": (c_int, [c_int]),
    "slab_autotune_stats": (c_int, [ctypes.POINTER(c_int)] * 4),
    "slab_factor_batched": (c_int, [c_int, ctypes.POINTER(SlabGrid), ctypes.POINTER(SlabCoeffs),
                                    ctypes.POINTER(c_int), ctypes.POINTER(SlabOpts), c_int, ctypes.POINTER(c_void_p)]),
    "slab_solve_batched": (c_int, [c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(c_int), ctypes.POINTER(c_void_p), ctypes.POINTER(c_int), c_int]),
    "slab_adjoint_batched": (c_int, [c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                     ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                     ctypes.POINTER(c_int), c_int]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libslab.so (building it first if needed).  Raises if it cannot be loaded: no fallback."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


def _strerror(status: int) -> str:
    try:
        return load(build_if_missing=False).slab_strerror(status).decode()
    except Exception:
        return f"status {status}"


def check(status: int, what: str = "", allow=()) -> int:
    if status != SLAB_OK and status not in allow:
        raise SlabError(status, what)
    return status
