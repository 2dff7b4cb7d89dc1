"""GB300-native PAKR: batched kinodynamic RRT expansion under an AO-x cost bound.

``pakr``      -- ctypes binding of the C ABI (include/pakr.h) over libpakr.so
``workloads`` -- seeded synthetic problem and tree generators
``_build``    -- in-tree nvcc build of libpakr.so for sm_103a
"""
from . import workloads  # noqa: F401

__all__ = ["pakr", "workloads"]
