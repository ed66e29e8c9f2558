"""GB300-native Loop-of-stencil-reduce (arXiv 1609.04567): one stencil sweep
fused with a global reduce, iterated on the device until a convergence test
passes.

The compute path is the C-ABI library ``libslr.so`` (hand-written sm_103a CUDA,
declared in ``include/slr.h``); ``paper_1609_04567_gb300.slr`` is its thin
ctypes binding.  Nothing here falls back to the CPU: without the compiled
library every call raises.
"""

__all__ = ["slr", "inputs"]
