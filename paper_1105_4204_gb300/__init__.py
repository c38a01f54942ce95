"""GB300-native trigonometric O(1) bilateral filter (Chaudhury, Sage, Unser).

The compute path is the CUDA library ``libbf.so`` (built from ``csrc/`` for
sm_103a by ``build.build()``); this package is its thin Python binding.
"""
from .api import (BOX, GAUSS, Batch, BilateralFunction, Plan, backward, bilateral,  # noqa: F401
                  backward_stack, forward, forward_host, forward_stack, forward_unfused,
                  forward_space_variant, fp32_pipe_rate, set_shape, tune)

__all__ = ["Plan", "forward", "forward_stack", "forward_host", "forward_unfused", "backward",
           "backward_stack", "bilateral", "tune", "set_shape", "fp32_pipe_rate", "forward_space_variant",
           "BilateralFunction", "Batch", "GAUSS", "BOX"]
