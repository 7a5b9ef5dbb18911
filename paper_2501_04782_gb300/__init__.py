"""GB300-native differentiable Gaussian rasterizer for GaussianVideo (arXiv 2501.04782).

Submodules:
  synth   -- seeded synthetic workloads (inputs only, no rendering arithmetic)
  gv      -- ctypes binding of the CUDA library libgv.so (the C-ABI in include/gv.h)
  render  -- torch.autograd.Function wrappers and the batched training helpers
"""
__all__ = ["synth", "gv", "render"]
