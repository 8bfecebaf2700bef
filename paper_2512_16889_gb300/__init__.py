"""GB300-native scattered-wave-function (SWF) Dirac solver.

The compute path is the CUDA library ``libswf.so`` (C ABI in ``include/swf.h``); ``swf`` is its
ctypes binding, ``workloads`` the seeded synthetic instance tables, ``build`` the nvcc build.
"""
from . import workloads  # noqa: F401
