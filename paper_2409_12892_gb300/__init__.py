"""GB300 (sm_103a) Levenberg-Marquardt / PCG hot path for 3D Gaussian Splatting.

The compute path lives in ``libgslm.so`` (hand-written CUDA, C ABI in
``include/gslm.h``); ``gslm`` is its thin Python binding.
"""
from .gslm import (Cache, Context, GslmError, Precond, load_library, padded_ld, to_soa, from_soa,  # noqa: F401
                   make_cameras, n_pixels, exported_symbols, kernel_launches, LIB_PATH)
