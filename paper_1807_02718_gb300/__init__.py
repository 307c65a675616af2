"""GB300-native fast-hybrid 2D wave scattering (frequency solves + recentred synthesis).

The compute path is libfh.so (CUDA kernels for sm_103a behind the C ABI in
include/fh.h); `fh` is its thin Python binding.  Build with build.build().
"""
from . import fh  # noqa: F401  (binding; the library loads on first call)

__all__ = ["fh"]
