"""GB300-native PDE-EPDiff LDDMM (arXiv 1807.04638): geodesic shooting, reduced
gradient and Gauss-Newton Hessian-vector products on one GPU.

The numerical work lives in the CUDA library ``lib/liblddmm.so`` (C ABI in
``include/lddmm.h``); ``Handle`` marshals torch tensors into it.  Build the
library with ``python -m paper_1807_04638_gb300.build``.
"""
from ._native import (  # noqa: F401
    LDDMM_BF16, LDDMM_F32, LDDMM_F64, LDDMM_GRAD_DISCRETE, LDDMM_GRAD_JACOBI, LDDMM_INTERP_CUBIC, LDDMM_INTERP_LINEAR, LDDMM_OPT_GD, LDDMM_OPT_GN,
    LDDMM_SPACE_L2, LDDMM_SPACE_V,
    Handle, LddmmError, apply_metric_noalloc, default_params, lib, make_grid, probe_fp64_fma, workspace_bytes,
)
