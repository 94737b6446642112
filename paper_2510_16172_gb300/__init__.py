"""GB300-native batched Fermat path solve (arXiv 2510.16172).

The CUDA library (``libfpt.so``, built by :mod:`paper_2510_16172_gb300.build`)
does all of the work; :mod:`paper_2510_16172_gb300.fpt` binds its C ABI
(include/fpt.h) and :mod:`paper_2510_16172_gb300.autograd` wraps solve and
backward in a ``torch.autograd.Function``.  :mod:`paper_2510_16172_gb300.scenes`
draws the seeded synthetic scenes.
"""

__all__ = ["build", "fpt", "scenes", "autograd"]
