"""GB300-native multilevel linearized-buckling solver (multigrid-preconditioned CG, stress
stiffness, coarse-grid buckling modes, adjoint sensitivities) behind the C-ABI of include/tobk.h.

The compute path is libtobk.so (hand-written CUDA for sm_103a); `binding` is a ctypes layer over
it.  There is no CPU fallback: using the solver without the built library raises."""
from .binding import (Solver, Batch, UNet, TobkError, load, launch_count, KERNEL_CLASSES, TOBK_FP64, TOBK_FP32_VCYCLE, TOBK_FIELD_U,  # noqa: F401
                      TOBK_FIELD_MODES, TOBK_FIELD_ADJOINT, TOBK_FIELD_ADJOINT_RHS, TOBK_FIELD_FINE_ADJOINT,
                      TOBK_FIELD_COARSE_ADJOINT, TOBK_FIELD_PROLONGATED, TOBK_E_ARG, EXPORTED)

__all__ = ["Solver", "Batch", "UNet", "TobkError", "load", "EXPORTED"]
