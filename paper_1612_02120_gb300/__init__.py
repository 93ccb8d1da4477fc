"""libmembrane: dense membrane-probability inference (arXiv 1612.02120, Sec. 2.1-2.2) on GB300.

The compute path is the CUDA library ``libmembrane.so`` (C ABI in include/membrane.h);
``membrane`` is its ctypes binding and ``build`` compiles it for sm_103a.
"""
from . import build, membrane  # noqa: F401

__all__ = ["build", "membrane"]
