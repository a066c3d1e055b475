"""GB300-native chi0 / eps^-1 hot path of the GW method (arXiv:1902.03837).

The computation lives in libchi0.so (CUDA, sm_103a) behind the C ABI of
include/chi0.h; ``paper_1902_03837_gb300.chi0`` is its ctypes binding.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchi0.so")


def build(force=False, verbose=False):
    from .buildlib import build as _build
    return _build(force=force, verbose=verbose)
