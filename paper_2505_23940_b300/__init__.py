"""B300-native fractional-step finite-volume / immersed-boundary time step.

The data-parallel hot path of Diff-FlowFSI (arXiv 2505.23940): convection-
diffusion predictor, pressure-Poisson projection, immersed-boundary direct
forcing with a regularised delta kernel and the rigid-body update, as
hand-written sm_103a CUDA kernels behind the C ABI of include/fs.h.
Python here only marshals arguments; there is no CPU fallback.
"""
from .fsstep import (CENTRAL2, FE, FP64, FREESLIP, INFLOW, MIXED, NOSLIP, OUTFLOW, PERIODIC,  # noqa: F401
                     PESKIN4, RK3, ROMA3, UPWIND1, FsError, Grid, check, lib)
from .workload import body_tensor, grid_from_workload  # noqa: F401
