"""Brute-force walk enumeration (Prop. power-of-adjacency; Sec. 3.2 for the
backtrack-downweighted weights). Pure Python; tiny graphs only. Test
infrastructure only."""
import numpy as np


def weighted_walk_counts(A, k, mu):
    """(q_k)_ij = sum over walks i = i_0, ..., i_k = j of (1 - mu)^{b}, where
    b counts the steps with i_l = i_{l+2} (Sec. 3.2). mu = 0 counts all walks,
    mu = 1 counts nonbacktracking walks only (0^0 = 1)."""
    n = A.shape[0]
    nbrs = [np.nonzero(A[i])[0].tolist() for i in range(n)]
    theta = 1.0 - mu
    Q = np.zeros((n, n))

    def rec(walk, weight):
        if len(walk) == k + 1:
            Q[walk[0], walk[-1]] += weight
            return
        for j in nbrs[walk[-1]]:
            w = weight
            if len(walk) >= 2 and j == walk[-2]:
                w = w * theta
            if w != 0.0:
                rec(walk + [j], w)

    for i in range(n):
        if k == 0:
            Q[i, i] = 1.0
        else:
            rec([i], 1.0)
    return Q
