"""GB300-native (sm_103a) dense-indirect EM of VOLDOR+ (arxiv 2104.06800).

The compute path is the CUDA library ``libvoldor_em.so`` (C ABI in
``include/voldor_em.h``); ``voldor`` is its ctypes binding and ``build``
compiles it in-tree.
"""
from . import voldor  # noqa: F401
from .voldor import load  # noqa: F401

__all__ = ["voldor", "load"]
