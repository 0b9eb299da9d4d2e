"""GB300-native EPIC imaging: C-ABI CUDA library (libepic.so) + thin Python binding.

The hot path (4+4-bit unpack -> gridding -> 2-D transform -> polarisation
products -> time accumulation, paper Sec. 2 Eq. 1-2) runs entirely in the
sm_103a kernels of libepic.so; this package only builds and calls it.
"""
from .epic import (  # noqa: F401
    ACCUMULATE, EXPORTED, PATHS, PATH_AUTO, PATH_DFTGEMM_FP16, PATH_FUSED_FP32, PATH_PLAIN_FP32, RESET,
    EpicError, Plan, Server, device_query, library_path, load,
)
from .buildlib import build  # noqa: F401
