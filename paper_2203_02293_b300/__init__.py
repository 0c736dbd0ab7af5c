"""B300-native column radiative transfer (improved two-stream + Thomas).

The computation lives in the CUDA library ``librt.so`` (C ABI in
``include/rt.h``); ``rt`` is its ctypes binding and ``solver`` wraps device
memory and a handle.  Importing ``solver`` needs torch; ``rt`` needs only the
built library.
"""
from . import rt  # noqa: F401

__all__ = ["rt"]
