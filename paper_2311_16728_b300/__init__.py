"""B300-native differentiable 3D-Gaussian rasterisation for Photo-SLAM-style
photorealistic mapping (arXiv 2311.16728, Sec. 3.3-3.4).

The compute lives in libgsr.so (hand-written CUDA for sm_103a behind the C ABI
of include/gsr.h); `_lib` binds it name for name and `raster` wraps it for
PyTorch tensors, autograd and CUDA graphs.  Importing this package raises if
libgsr.so has not been built: there is no CPU or library fallback.
"""
from . import _lib
from ._lib import GsrError
from .raster import (LAMBDA_DSSIM, PYRAMID_LEVELS, STAGES, Adam, AdamConfig, Gaussians, MappingStep, RasterizeGaussians,
                     ViewBuffers, camera_at_level, camera_from, camera_struct, ensure_capacity, n_tiles, psnr,
                     permuted, pyramid, rasterize, spatial_order, tiling_struct)
from .pose import PoseRefiner, so3_exp

__all__ = ["_lib", "GsrError", "LAMBDA_DSSIM", "PYRAMID_LEVELS", "STAGES", "Adam", "AdamConfig", "Gaussians", "MappingStep",
           "RasterizeGaussians", "ViewBuffers", "camera_at_level", "camera_from", "camera_struct", "ensure_capacity",
           "n_tiles", "psnr", "pyramid", "rasterize", "tiling_struct", "PoseRefiner", "so3_exp",
           "spatial_order", "permuted"]
