"""GB300 (sm_103a) library for the data-parallel hot path of arXiv:2307.07999:
boost-invariant SU(3) Glasma leapfrog + colored particle-in-cell Wong push +
momentum-broadening estimators (kappa, qhat).

The compute runs in libglasma.so (CUDA C ABI, include/glasma.h).  This package
only marshals arguments: ctypes structures mirroring the C structs, thin
wrappers with the C names, and PyTorch for device workspaces and streams.
There is no CPU fallback: importing the binding fails loudly if the library
has not been built.
"""
from ._lib import (  # noqa: F401
    GLASMA_FP32,
    GLASMA_FP64,
    CpicParams,
    GlasmaError,
    GlasmaParams,
    lib,
)
from .api import (  # noqa: F401
    CPIC,
    Batch,
    Correlators,
    Glasma,
    HBARC,
    WarmStartNet,
    ic_dataset,
    init_warm,
    broadening_accumulate,
    broadening_transport,
    cpic_create,
    cpic_init,
    cpic_push,
    cpic_push_many,
    push_many,
    anisotropy,
    pool_broadening,
    field_tile_shape,
    field_tile_variants,
    glasma_create,
    glasma_init,
    glasma_step,
    kappa_qhat,
)
