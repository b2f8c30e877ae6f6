"""Error measures of the GPU parity tests (CUDA path against the CPU FP64
oracle), per output column:

  norm-wise     |got - want|_2 / |want|_2
  element-wise  max_i |got_i - want_i| / max_i |want_i|

`relerr` returns the larger of the two, so every parity assertion bounds
both: a wrong value on a low-magnitude row (an isolated node, a leaf, the
tail of a diffusion profile) that the norm-wise measure would absorb still
has to sit within the tolerance of the column's largest entry."""
import numpy as np


def _cols(a):
    a = np.asarray(a, dtype=np.float64)
    return a[:, None] if a.ndim == 1 else a.reshape(a.shape[0], -1)


def normerr(got, want):
    g, w = _cols(got), _cols(want)
    return float((np.linalg.norm(g - w, axis=0) / np.maximum(np.linalg.norm(w, axis=0), 1e-300)).max())


def elemerr(got, want):
    g, w = _cols(got), _cols(want)
    return float((np.abs(g - w).max(axis=0) / np.maximum(np.abs(w).max(axis=0), 1e-300)).max())


def relerr(got, want):
    return max(normerr(got, want), elemerr(got, want))
