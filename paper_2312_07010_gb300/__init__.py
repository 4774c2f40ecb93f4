"""GB300-native RLB-MIE-FD stepper for the Allen-Cahn equation (arXiv:2312.07010).

The compute path is ``libacs.so`` (hand-written sm_103a CUDA behind the C ABI of
``include/acs.h``); this package only marshals arguments to it.  Importing the
package does not load the library; the first call that needs it does, and fails
loudly when it has not been built (``paper_2312_07010_gb300.build.build()``).
"""
from . import build
from ._lib import (ACS_BC_DIRICHLET, ACS_BC_NEUMANN, ACS_BC_PERIODIC, ACS_E_CUDA, ACS_E_INVAL,
                   ACS_E_NOMEM, ACS_E_NONFINITE, ACS_E_STATE, ACS_E_TIMEOUT, ACS_E_UNSUPPORTED, ACS_F32, ACS_F64,
                   ACS_KERNEL_AUTO, ACS_KERNEL_NAIVE, ACS_KERNEL_TEMPORAL, ACS_KERNEL_TILED,
                   ACS_ROOT_NEWTON, ACS_ROOT_NONE, ACS_ROOT_SERIES, ACS_SCHEME_FEX_FD, ACS_SCHEME_RLB_MIE_FD, SIGNATURES, AcsError, check, lib,
                   lib_path, strerror)

__all__ = [
    "build", "lib", "lib_path", "strerror", "check", "AcsError", "SIGNATURES",
    "ACS_BC_PERIODIC", "ACS_BC_NEUMANN", "ACS_BC_DIRICHLET", "ACS_F32", "ACS_F64",
    "ACS_E_INVAL", "ACS_E_CUDA", "ACS_E_NOMEM", "ACS_E_TIMEOUT", "ACS_E_NONFINITE", "ACS_E_STATE",
    "ACS_E_UNSUPPORTED",
    "ACS_KERNEL_AUTO", "ACS_KERNEL_NAIVE", "ACS_KERNEL_TILED", "ACS_KERNEL_TEMPORAL",
    "ACS_SCHEME_RLB_MIE_FD", "ACS_SCHEME_FEX_FD", "ACS_ROOT_NEWTON", "ACS_ROOT_SERIES", "ACS_ROOT_NONE",
    "AllenCahn", "AllenCahnFunction", "allen_cahn", "Batch", "Lines", "Pipeline", "dt_max",
]


def __getattr__(name):
    # torch-dependent front ends are imported on first use
    if name in ("AllenCahn", "AllenCahnFunction", "allen_cahn", "dt_max"):
        from . import stepper
        return getattr(stepper, name)
    if name == "Batch":
        from . import batch
        return batch.Batch
    if name == "Lines":
        from . import lines
        return lines.Lines
    if name == "Pipeline":
        from . import pipeline
        return pipeline.Pipeline
    raise AttributeError(name)
