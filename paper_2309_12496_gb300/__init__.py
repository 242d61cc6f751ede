"""GB300-native Cherenkov photon propagator (sm_103a CUDA + C ABI).

* ``workloads`` -- seeded synthetic scenes and tracks (inputs only);
* ``rich``      -- the Python binding of the C ABI in ``include/rich.h``;
* ``build``     -- compiles ``librich.so`` in-tree for sm_103a.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "rich", "build"]
