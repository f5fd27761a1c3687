"""Compressed out-of-core 3D stencil sweeps on one GB300 (sm_103a).

The compute path is the CUDA library ``liboocs.so`` built from ``csrc/`` and
called through the C ABI in ``include/oocs.h``; ``oocs.py`` is its ctypes
binding.  Nothing in this package computes on the CPU.
"""
from .oocs import *  # noqa: F401,F403
from .oocs import lib, library_path, OutOfCoreStencil, OOCSError, make_desc  # noqa: F401

__version__ = "0.1"
