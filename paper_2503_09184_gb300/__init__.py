"""GB300-native encrypted sparse matrix multiplication (RNS BFV).

The CUDA library (libsfhe.so, include/sfhe.h) does every step of the
computation; `sfhe` is its ctypes binding and `api` a convenience layer
that keeps ciphertexts in torch device tensors.
"""
from . import sfhe  # noqa: F401
