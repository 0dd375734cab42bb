"""GB300 (sm_103a) implementation of the Flow Fields patch-matching loop.

arXiv 1703.02563 (Bailer, Taetz, Stricker): WHT features, exact seeding,
raster-order propagation with random search over a coarse-to-fine scale
space, and the forward/backward consistency check, as hand-written CUDA
behind the C ABI in include/ff.h.  ``ff`` is the Python binding.
"""
from . import ff  # noqa: F401
