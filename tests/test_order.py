"""Reverse Cuthill-McKee relabelling (wl_rcm_order, host code; the option
reorder = 2 of wl_build). Checked against what the ordering must do, not
against an implementation: a permutation, components on contiguous label
ranges, and the bandwidth of a randomly shuffled grid brought back to about its
width (comparable to scipy's reverse_cuthill_mckee); deterministic."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, reverse_cuthill_mckee

import wlgen
from paper_2601_11338_gb300 import wl


def _shuffle(g, seed):
    rng = np.random.default_rng(seed)
    p = rng.permutation(g.n)  # new label of old node i is p[i]
    A = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    P = sp.csr_matrix((np.ones(g.n), (p, np.arange(g.n))), shape=(g.n, g.n))
    B = (P @ A @ P.T).tocsr()
    B.sort_indices()
    return B.indptr.astype(np.int32), B.indices.astype(np.int32), B


def _bandwidth(rp, ci, iperm):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return int(np.abs(iperm[rows] - iperm[ci]).max()) if len(ci) else 0


def _check_perm(perm, n):
    assert perm.dtype == np.int32 and perm.shape == (n,)
    assert np.array_equal(np.sort(perm), np.arange(n))


def test_shuffled_grid_bandwidth_is_restored():
    r, c = 30, 50
    rp, ci, B = _shuffle(wlgen.grid2d(r, c), 5)
    n = r * c
    perm = wl.wl_rcm_order(rp, ci, n)
    _check_perm(perm, n)
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    ours = _bandwidth(rp, ci, iperm)
    sperm = reverse_cuthill_mckee(B, symmetric_mode=True)
    siperm = np.empty(n, np.int64)
    siperm[sperm] = np.arange(n)
    theirs = _bandwidth(rp, ci, siperm)
    shuffled = _bandwidth(rp, ci, np.arange(n))
    assert shuffled > 10 * min(r, c)
    assert ours <= 2 * min(r, c) + 2, ours
    assert ours <= 1.5 * theirs + 2, (ours, theirs)


def test_components_get_contiguous_labels_and_isolated_nodes_are_kept():
    # two ER blocks, a path and isolated nodes, interleaved by a shuffle
    a = wlgen.erdos_renyi(200, 6, 1)
    b = wlgen.erdos_renyi(150, 5, 2)
    A = sp.block_diag([sp.csr_matrix((np.ones(a.nnz), a.col_idx, a.row_ptr), shape=(a.n, a.n)),
                       sp.csr_matrix((np.ones(b.nnz), b.col_idx, b.row_ptr), shape=(b.n, b.n)),
                       sp.diags([np.ones(9), np.ones(9)], [-1, 1], shape=(10, 10)),
                       sp.csr_matrix((7, 7))]).tocsr()
    n = A.shape[0]
    g = wlgen.CSR(n, A.indptr.astype(np.int64), A.indices.astype(np.int32))
    rp, ci, B = _shuffle(g, 9)
    perm = wl.wl_rcm_order(rp, ci, n)
    _check_perm(perm, n)
    _, lab = connected_components(B, directed=False)
    comp_of_new = lab[perm]
    # each component's new labels form one run
    changes = np.count_nonzero(comp_of_new[1:] != comp_of_new[:-1])
    assert changes == len(np.unique(lab)) - 1
    assert np.array_equal(perm, wl.wl_rcm_order(rp, ci, n))  # deterministic


def test_edge_cases():
    assert wl.wl_rcm_order(np.zeros(1, np.int32), np.zeros(0, np.int32), 0).shape == (0,)
    _check_perm(wl.wl_rcm_order(np.zeros(6, np.int32), np.zeros(0, np.int32), 5), 5)
    g = wlgen.chung_lu(5000, seed=3)
    _check_perm(wl.wl_rcm_order(g.row_ptr.astype(np.int32), g.col_idx, g.n), g.n)
    with pytest.raises(wl.WLError):
        wl.wl_rcm_order(np.zeros(1, np.int32), np.zeros(0, np.int32), -1)
