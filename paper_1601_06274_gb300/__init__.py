"""GB300-native dense stereo matching (arXiv 1601.06274): census cost volume,
Dual MM with hierarchical minorants, non-linear primal-dual refinement.

The compute lives in libdm.so (CUDA, sm_103a; C ABI in include/dm.h);
``dm`` is its Python binding and ``synthetic`` the seeded input generator.
"""

__all__ = ["dm", "synthetic", "build"]
