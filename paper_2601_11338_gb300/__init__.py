"""GB300-native walk-based Laplacians (Arrigo and Durastante, arXiv 2601.11338).

The compute path is libwl.so (hand-written CUDA for sm_103a, C ABI in
include/wl.h); `wl` is its ctypes binding and `api` a convenience layer on
top of it. Importing this package does not load the CUDA library; the first
call does, and fails loudly if it is missing.
"""
from . import build  # noqa: F401
