"""lfbp: light-field backprojection arrays H' from PSF arrays H on one GB300.

The H -> H' construction of arXiv 2003.09133 (Sec. 3, Eqs. 4-9) as
hand-written sm_103a kernels behind a C-ABI (include/lfbp.h), with a thin
ctypes binding and a torch.autograd.Function whose backward is the adjoint
gather.  PyTorch supplies device memory and streams only.
"""
from ._lib import (F16, F32, MAP_PAPER_WINDOW, MAP_TRANSPOSE, LfbpError, Plan, adjoint,
                   backproject_array, backproject_batched, lib_path, load, sync_status)
from .autograd import LFBackproject, backprojection_array

__all__ = [
    "Plan", "backproject_array", "backproject_batched", "adjoint", "sync_status", "load",
    "lib_path", "LfbpError", "LFBackproject", "backprojection_array", "MAP_TRANSPOSE",
    "MAP_PAPER_WINDOW", "F32", "F16",
]
