"""GB300 (sm_103a) solver for the 3D Helmholtz equation with Sommerfeld absorbing boundaries:
compact 4th/6th-order schemes, EigT (and PFFT) preconditioners that include the absorbing boundary,
restarted/flexible GMRES (arXiv 2602.07711).

The compute path is the C-ABI library libhelm.so (include/helm.h), built in-tree by build.py.
This package only marshals arguments (torch tensors, streams) into that library.
"""
from .helm import (HELM_C64, HELM_C128, HELM_PREC_FP32, HELM_PREC_TF32, HELM_PREC_TF32X3, HELM_PREC_BF16, HELM_PREC_FP16,
                   HELM_PRECOND_EIGT,
                   HELM_PRECOND_NONE, HELM_PRECOND_PFFT, HELM_PRECOND_FFT2, HELM_CLOSURE_THREE_POINT,
                   HELM_CLOSURE_HIGH_ORDER, Batch, HelmError, Net, Solver, lib, library_path, solve_batched)

__all__ = ["Solver", "Net", "Batch", "solve_batched", "HelmError", "lib", "library_path", "HELM_C64", "HELM_C128",
           "HELM_PREC_FP32", "HELM_PREC_TF32", "HELM_PREC_TF32X3", "HELM_PREC_BF16", "HELM_PREC_FP16",
           "HELM_PRECOND_NONE", "HELM_PRECOND_EIGT", "HELM_PRECOND_PFFT", "HELM_PRECOND_FFT2",
           "HELM_CLOSURE_THREE_POINT", "HELM_CLOSURE_HIGH_ORDER"]
