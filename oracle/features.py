"""Local node features for the warm-start network, dense FP64 (test
infrastructure only). Per node i:

  f0 = log(1 + d_i)                 degree
  f1 = log(1 + (A d)_i)             neighbour-degree sum
  f2 = log(1 + (A^3)_ii / 2)        triangles through i
  f3 = log(1 + (A d - d)_i)         2-hop count, read as the number of
                                    nonbacktracking walks of length 2 from i,
                                    (p_2(A) 1)_i with p_2 = A^2 - D (Eq. Br)
"""
import numpy as np


def raw_features(A):
    d = A.sum(axis=1)
    Ad = A @ d
    tri = np.diag(A @ A @ A) / 2.0
    return np.stack([np.log1p(d), np.log1p(Ad), np.log1p(tri), np.log1p(Ad - d)], axis=1)


def triangles_by_intersection(row_ptr, col_idx, n):
    """Triangle count per node by sorted-list intersection (independent of A^3)."""
    nb = [set(col_idx[row_ptr[i]:row_ptr[i + 1]].tolist()) for i in range(n)]
    t = np.zeros(n)
    for i in range(n):
        for j in nb[i]:
            if j > i:
                for k in nb[i] & nb[j]:
                    if k > j:
                        t[i] += 1; t[j] += 1; t[k] += 1
    return t
