"""DDGS-CT DRR splatting on GB300 (sm_103a): forward and backward rendering of
direction-disentangled Gaussian clouds behind a C ABI (include/ddgs.h).

Modules:
  binding    -- ctypes marshalling over libddgs.so, workspace, autograd Function
  build      -- nvcc build of libddgs.so (sm_103a only), in-tree
  synthetic  -- seeded synthetic inputs (phantoms, clouds, poses); no renderer math
"""
from . import build, synthetic  # noqa: F401

__all__ = ["build", "synthetic", "binding"]
