"""GB300-native masked 4D Gaussian splatting rasterizer (4DGS-1K, arXiv 2503.16422).

Modules:
  build   compiles the CUDA library libfdgs.so for sm_103a (in-tree)
  fdgs    ctypes binding of the C ABI (include/fdgs.h) and the autograd render function
  scenes  seeded synthetic scenes, cameras and key-frame masks
"""
__all__ = ["build", "fdgs", "scenes"]
