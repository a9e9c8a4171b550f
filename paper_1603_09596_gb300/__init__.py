"""GB300-native batched kd-GeRaF search (Avrithis, Emiris, Samaras, arXiv 1603.09596).

The compute path is the CUDA library ``libgf.so`` (C ABI in ``include/gf.h``); ``gf`` is its
Python binding.  Importing the binding requires the compiled library.
"""
from . import _build  # noqa: F401
from .gf import *  # noqa: F401,F403
from .gf import Forest, GFError, lib  # noqa: F401
