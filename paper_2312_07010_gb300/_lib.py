"""ctypes binding of ``libacs.so`` (declared in ``include/acs.h``).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

ACS_BC_PERIODIC, ACS_BC_NEUMANN, ACS_BC_DIRICHLET = 0, 1, 2
ACS_F32, ACS_F64 = 0, 1
ACS_OK = 0
ACS_WARN_MP_CONDITION, ACS_WARN_ENERGY_CONDITION = 1, 2
ACS_E_INVAL, ACS_E_CUDA, ACS_E_NOMEM, ACS_E_TIMEOUT = -1, -2, -3, -4
ACS_E_NONFINITE, ACS_E_STATE, ACS_E_UNSUPPORTED = -5, -6, -7
ACS_KERNEL_AUTO, ACS_KERNEL_NAIVE, ACS_KERNEL_TILED, ACS_KERNEL_TEMPORAL, ACS_KERNEL_LB = 0, 1, 2, 3, 4
ACS_SCHEME_RLB_MIE_FD, ACS_SCHEME_FEX_FD = 0, 1
ACS_ROOT_NEWTON, ACS_ROOT_SERIES, ACS_ROOT_NONE = 0, 1, 2

# every function include/acs.h declares: name -> (restype, argtypes)
_c = ctypes
_vp = _c.c_void_p
_i64 = _c.c_int64
_dp = _c.POINTER(_c.c_double)
_i64p = _c.POINTER(_c.c_int64)
SIGNATURES = {
    "acs_create": (_c.c_int, [_c.c_int, _i64p, _c.c_double, _c.c_double, _c.c_double, _c.c_int, _c.c_int,
                              _c.POINTER(_vp)]),
    "acs_work_bytes": (_c.c_size_t, [_vp]),
    "acs_bind": (_c.c_int, [_vp, _vp, _vp, _c.c_size_t, _vp]),
    "acs_set_state": (_c.c_int, [_vp, _vp]),
    "acs_set_state_host": (_c.c_int, [_vp, _vp]),
    "acs_get_state_host": (_c.c_int, [_vp, _vp]),
    "acs_set_scheme": (_c.c_int, [_vp, _c.c_int]),
    "acs_set_kernel": (_c.c_int, [_vp, _c.c_int, _c.c_int]),
    "acs_get_kernel": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "acs_get_root": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "acs_num_variants": (_c.c_int, []),
    "acs_set_variant": (_c.c_int, [_vp, _c.c_int, _c.c_int]),
    "acs_get_variant": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "acs_autotune": (_c.c_int, [_vp, _dp]),
    "acs_step": (_c.c_int, [_vp, _i64]),
    "acs_steps_done": (_i64, [_vp]),
    "acs_energy": (_c.c_int, [_vp, _dp]),
    "acs_maxnorm": (_c.c_int, [_vp, _dp]),
    "acs_phase_volume": (_c.c_int, [_vp, _dp]),
    "acs_observe_async": (_c.c_int, [_vp, _vp]),
    "acs_run_logged": (_c.c_int, [_vp, _i64, _i64, _dp, _dp]),
    "acs_grad_work_bytes": (_c.c_size_t, [_vp, _i64, _i64]),
    "acs_grad_bind": (_c.c_int, [_vp, _vp, _c.c_size_t, _i64, _i64]),
    "acs_grad": (_c.c_int, [_vp, _vp, _vp, _dp]),
    "acs_observe_noalloc": (_c.c_int, [_c.c_int, _i64p, _c.c_double, _c.c_double, _c.c_int, _c.c_int, _vp,
                                       _vp, _vp]),
    "acs_sync": (_c.c_int, [_vp]),
    "acs_dt_max": (_c.c_int, [_c.c_int, _c.c_double, _c.c_double, _dp, _dp]),
    "acs_strerror": (_c.c_char_p, [_c.c_int]),
    "acs_version": (_c.c_char_p, []),
    "acs_destroy": (None, [_vp]),
    "acs_lb_bytes": (_c.c_size_t, [_vp]),
    "acs_lb_bind": (_c.c_int, [_vp, _vp, _c.c_size_t, _c.c_double]),
    "acs_batch_create": (_c.c_int, [_c.c_int, _i64p, _dp, _dp, _dp, _c.POINTER(_c.c_int), _c.c_int,
                                    _c.POINTER(_vp)]),
    "acs_batch_numel": (_c.c_size_t, [_vp]),
    "acs_batch_offsets": (_c.c_int, [_vp, _i64p]),
    "acs_batch_row_strides": (_c.c_int, [_vp, _i64p]),
    "acs_batch_work_bytes": (_c.c_size_t, [_vp]),
    "acs_batch_bind": (_c.c_int, [_vp, _vp, _vp, _c.c_size_t, _vp]),
    "acs_batch_step": (_c.c_int, [_vp, _i64]),
    "acs_batch_set_config": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int]),
    "acs_batch_get_config": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "acs_batch_autotune": (_c.c_int, [_vp, _dp]),
    "acs_batch_set_temporal": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int]),
    "acs_batch_get_temporal": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "acs_batch_observe": (_c.c_int, [_vp, _dp, _dp]),
    "acs_batch_inject_fault": (_c.c_int, [_vp, _c.c_int]),
    "acs_batch_destroy": (None, [_vp]),
    "acs_lines_create": (_c.c_int, [_c.c_int, _i64p, _dp, _dp, _dp, _c.POINTER(_c.c_int), _c.c_int,
                                    _c.POINTER(_vp)]),
    "acs_lines_numel": (_c.c_size_t, [_vp]),
    "acs_lines_offsets": (_c.c_int, [_vp, _i64p]),
    "acs_lines_work_bytes": (_c.c_size_t, [_vp]),
    "acs_lines_bind": (_c.c_int, [_vp, _vp, _vp, _c.c_size_t, _vp]),
    "acs_lines_step": (_c.c_int, [_vp, _i64]),
    "acs_lines_observe": (_c.c_int, [_vp, _dp, _dp]),
    "acs_lines_destroy": (None, [_vp]),
    "acs_pipe_create": (_c.c_int, [_c.c_int, _i64p, _c.c_double, _c.c_double, _c.c_double, _c.c_int, _c.c_int,
                                   _c.c_int, _c.POINTER(_vp)]),
    "acs_pipe_bytes": (_c.c_size_t, [_vp]),
    "acs_pipe_bind": (_c.c_int, [_vp, _vp, _c.c_size_t, _vp]),
    "acs_pipe_context": (_vp, [_vp, _c.c_int]),
    "acs_pipe_submit": (_c.c_int, [_vp, _vp, _vp, _i64, _i64, _dp]),
    "acs_pipe_wait": (_c.c_int, [_vp]),
    "acs_pipe_destroy": (None, [_vp]),
}

_lib = None


class AcsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else f"{strerror(status)} ({status})")


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libacs.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise ImportError(f"libacs.so is not built ({path}); run paper_2312_07010_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().acs_strerror(int(status)).decode()


def check(status: int, what: str = "") -> int:
    """Raise AcsError for a negative status; return warnings (> 0) unchanged."""
    if status < 0:
        raise AcsError(status, what)
    return status
