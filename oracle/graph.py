"""Dense views of a simple undirected graph (Sec. 2, Defs. adjacency and
undirected_laplacian). Test infrastructure only (see the package header)."""
import numpy as np


def dense_adjacency(row_ptr, col_idx, n):
    """A_ij = 1 if (i, j) is an edge, else 0 (Def. adjacency)."""
    A = np.zeros((n, n), dtype=np.float64)
    row_ptr = np.asarray(row_ptr)
    for i in range(n):
        A[i, col_idx[row_ptr[i]:row_ptr[i + 1]]] = 1.0
    return A


def degree_vector(A):
    """d = A 1, the diagonal of the degree matrix D (Sec. 2.1)."""
    return A.sum(axis=1)


def combinatorial_laplacian(A):
    """L = D - A (Def. undirected_laplacian)."""
    return np.diag(degree_vector(A)) - A
