"""GB300-native differentiable packed-mesh rasterizer with soft blends.

The compute path is the C-ABI library ``libmeshrast.so`` (hand-written CUDA
for sm_103a, declared in ``include/meshrast.h``).  ``paper_2007_08501_gb300.ops``
is its thin Python binding; ``paper_2007_08501_gb300.autograd`` wraps it in
``torch.autograd.Function``s.  Importing this package loads nothing: the
library is opened on first use, and a missing library is an error, never a
fallback.
"""
__all__ = ["workloads"]
