"""HiGS on GB300: hierarchically tiled 3D Gaussian Splatting render path
(arxiv 2606.00352) as sm_103a CUDA kernels behind a C ABI (include/higs.h).

Submodules:
  higs    - ctypes binding of libhigs.so (no CPU fallback)
  scenes  - seeded synthetic scenes and cameras (inputs only)
  build   - nvcc build of libhigs.so for sm_103a
"""
__all__ = ["higs", "scenes", "build"]
