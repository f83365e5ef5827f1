"""GB300-native (sm_103a) differentiable equirectangular Gaussian splatting: the hot path of OmniGS (arXiv 2404.03202).

The computation lives in the CUDA library `libomnigs.so` (C ABI in include/omnigs.h, sources in csrc/). This package
binds it (`_cabi`, same names as the C entry points) and chains the calls for a frame (`rasterizer`). Importing the
package fails if the library has not been built: there is no CPU fallback.
"""
from . import _cabi
from ._cabi import OmnigsError, make_config
from .rasterizer import OmniRender, Rasterizer, Settings, render

_cabi.load()

__all__ = ["OmnigsError", "OmniRender", "Rasterizer", "Settings", "make_config", "render"]
