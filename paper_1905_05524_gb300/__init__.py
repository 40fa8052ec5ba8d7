"""GB300-native ADER-DG hot path (Krenz, Rannabauer, Bader, arXiv 1905.05524).

The computation lives in ``_build/libaderdg.so`` (hand-written sm_103a CUDA
behind the C ABI of ``include/aderdg.h``); ``solver`` is a thin PyTorch/ctypes
front end.  There is no CPU fallback: using the solver without the built
library raises.
"""
from . import _lib  # noqa: F401

__all__ = ["_lib"]
