"""GB300-native light-field sampling library (LumiPath, arXiv 1903.03837).

The hot path (ray/sphere hits, inverse spherical-Fibonacci 5-NN, tent filter
weights, 25-tap gather-blend and its backward scatter) runs in hand-written
sm_103a CUDA kernels behind a C ABI (include/lumipath.h, liblumipath.so).
``lumipath`` is the ctypes binding under the C names; ``torch_api`` the
tensor-level API; ``autotune`` picks launch shapes. There is no CPU path.
"""
from . import build, lumipath  # noqa: F401

__all__ = ["build", "lumipath"]
