"""GB300-native (sm_103a) HAVSampler: hierarchical adaptive voxel-guided point
sampling (arXiv 2305.14306) as hand-written CUDA behind a C ABI.

* ``hav``     -- the Python binding of libhav.so (include/hav.h)
* ``scenes``  -- seeded synthetic inputs shaped like the paper's workloads
* ``build``   -- nvcc build of libhav.so for sm_103a
"""
from . import scenes  # noqa: F401

__all__ = ["hav", "scenes", "build"]
