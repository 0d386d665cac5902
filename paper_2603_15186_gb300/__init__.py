"""GB300-native renderer of hierarchical 3D Gaussian Splatting scenes.

The render path (level-of-detail cut, EWA projection with SH colour, tile
binning by duplicated keys and a radix sort, front-to-back compositing) runs
in the hand-written CUDA kernels of libngs.so behind the C ABI of
include/ngs.h; ``Renderer`` marshals arguments to it."""
from ._lib import NgsError, EXPORTS  # noqa: F401
from .renderer import Renderer, Server, camera_struct, camera_array  # noqa: F401

__all__ = ["Renderer", "Server", "NgsError", "camera_struct", "camera_array", "EXPORTS"]
