"""GB300-native (sm_103a) differentiable tile rasterizer for quadric Gaussian primitives
(Quadratic Gaussian Splatting, arXiv 2411.16392).

Modules:
  build    - compiles csrc/*.cu into libqgs.so (in-tree)
  _lib     - ctypes declarations of the C ABI in include/qgs.h
  render   - Rasterizer (one qgs_ctx) and the QGSRender autograd.Function
  scenes   - seeded synthetic scenes and cameras (inputs only)
"""
__all__ = ["build", "render", "scenes"]
