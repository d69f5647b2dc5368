"""B300-native contourlet video codec (CVC, arXiv:1510.00561) hot path.

The compute lives in libcvc.so (CUDA, sm_103a) behind the C ABI of
include/cvc.h; this package marshals torch tensors into it.
"""
from ._lib import CvcError  # noqa: F401

_LAZY = ("Codec", "Batch", "Server", "CtPlan", "ct_layout", "modulus", "kernel_launches", "drop_levels", "Deflater")


def __getattr__(name):
    # the torch-facing front end is imported on first use, so that light
    # submodules (the synthetic input generator) import without torch
    if name in _LAZY:
        from . import codec
        return getattr(codec, name)
    raise AttributeError(name)
