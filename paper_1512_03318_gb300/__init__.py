"""GB300 (sm_103a) hot path of two-site DMRG on a cylinder in mixed real and momentum space
(arXiv:1512.03318): Python binding of libmrdmrg (see include/mrdmrg.h).

The binding only marshals arguments: every step runs in the library's CUDA kernels (or its
host MPO builder). Importing this package never falls back to another implementation: if
the shared library is missing, `lib()` raises.
"""
from .binding import (  # noqa: F401
    DMRG, MRD_BASIS_MIXED, MRD_BASIS_MIXED_REAL, MRD_BASIS_REAL, MRD_PREC_BF16X3, MRD_PREC_FF, MRD_PREC_FP64, MRD_PREC_TF32, MRD_OPT_AUTOTUNE,
    MRD_OPT_GRAPH, MRD_OPT_PER_TASK_LAUNCH, MRD_OPT_WAIT_LIMIT_US, MRD_OPT_REAL, MRD_DMRG_OPT_ENV_FP32, MRD_DMRG_OPT_REAL, MRD_DMRG_OPT_SVD_PRESWEEPS,
    MRD_SVD_F32_F64,
    MRD_SVD_F32_FF, MRD_SVD_F64, MRD_SVD_FF, Context, Heff, MPO, MrdError, launch_count, lib, lib_path)
