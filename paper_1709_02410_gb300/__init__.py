"""GB300 (sm_103a) library for the hot path of rigid-multiblob Brownian
dynamics above a no-slip wall (Sprinkle, Balboa Usabiaga, Patankar, Donev,
"Large Scale Brownian Dynamics of Confined Suspensions of Rigid Particles").

The computation lives in librpbd.so (C ABI in include/rpbd.h, CUDA kernels
in csrc/).  This package is a thin binding: torch tensors supply device
memory and streams, and every call goes straight to the library.
"""
from .api import Handle, RpbdError, F32, F64  # noqa: F401
from ._native import Forces, StepParams  # noqa: F401
