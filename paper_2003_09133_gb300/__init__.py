"""lfbp: light-field backprojection arrays H' from PSF arrays H on one GB300.

The H -> H' construction of arXiv 2003.09133 (Sec. 4, Eqs. 4-9) as
hand-written sm_103a kernels behind a C-ABI (include/lfbp.h), with a thin
ctypes binding and a torch.autograd.Function whose backward is the adjoint
gather.  PyTorch supplies device memory and streams only.
"""
from ._lib import (F16, F32, MAP_PAPER_WINDOW, MAP_TRANSPOSE, LfbpError, Plan, adjoint,
                   backproject_array, backproject_array_host, backproject_batched,
                   backproject_volume_from_h, backproject_volume_grad, forward_project,
                   lib_path, load, rl_normaliser, rl_step, sync_status, tune_batched)
from ._lib import backproject_volume as backproject_volume_raw
from .autograd import (LFBackproject, LFBackprojectVolume, backprojection_array,
                       backproject_volume)

__all__ = [
    "Plan", "backproject_array", "backproject_batched", "adjoint", "sync_status", "load",
    "lib_path", "LfbpError", "LFBackproject", "backprojection_array", "MAP_TRANSPOSE",
    "MAP_PAPER_WINDOW", "F32", "F16", "LFBackprojectVolume", "backproject_volume",
    "backproject_volume_raw", "backproject_volume_grad", "forward_project",
    "backproject_array_host", "tune_batched", "backproject_volume_from_h", "rl_step",
    "rl_normaliser",
]
