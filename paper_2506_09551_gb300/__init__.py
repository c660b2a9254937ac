"""GB300-native multi-shifted BiCG for Kramers-Heisenberg (RIXS) response functions.

The compute path is the CUDA library libmsbicg (C ABI in include/msbicg.h);
`native` is its ctypes binding and `api` marshals torch tensors / numpy
arrays into it.  PyTorch is used only for device memory and streams.
"""
from . import native  # noqa: F401

__all__ = ["native", "api", "build"]
