"""Seeded synthetic inputs for the walk-Laplacian workloads.

This module generates inputs only: graphs as simple undirected 0/1 CSR
adjacencies (symmetric, zero diagonal, sorted rows), Gaussian right-hand-side
blocks and point sources. It holds none of the method's arithmetic, so the
CPU oracle and the CUDA library can both consume its output without sharing
any computation.

Every generator is deterministic in its seed. Large graphs (R-MAT, Chung-Lu,
CSR assembly) use the small C helper `_gen.c`, built by `build_helper()`;
its randomness is a counter-based hash, so results do not depend on thread
count or CPU architecture. Small generators use numpy's PCG64.

The graphs are synthetic stand-ins for the paper's SuiteSparse networks
(Sec. 5, Table 1), which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_gen.c")
_LIB_PATH = os.path.join(_HERE, "libwlgen.so")
_lib = None


@dataclass
class CSR:
    """Simple undirected graph as a 0/1 CSR adjacency (values implicit)."""

    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col_idx: np.ndarray  # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def build_helper(force: bool = False) -> str:
    """Compile the C helper in-tree (gcc, OpenMP, no architecture flags)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_helper()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, i32p, i64p, f64p = (
            ctypes.c_int64,
            ctypes.c_uint64,
            ctypes.POINTER(ctypes.c_int32),
            ctypes.POINTER(ctypes.c_int64),
            ctypes.POINTER(ctypes.c_double),
        )
        lib.wlgen_rmat_edges.argtypes = [ctypes.c_int, i64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, u64, i32p, i32p]
        lib.wlgen_permutation.argtypes = [i64, u64, i32p]
        lib.wlgen_relabel.argtypes = [i64, i32p, i32p, i32p]
        lib.wlgen_chung_lu_edges.argtypes = [i64, f64p, i32p, u64, i64, i32p, i32p, i64p]
        lib.wlgen_csr_count.argtypes = [i64, i64, i32p, i32p, i64p, i64p]
        lib.wlgen_csr_fill.argtypes = [i64, i64, i32p, i32p, i64p, i32p, i64p]
        lib.wlgen_uniform.argtypes = [i64, u64, u64, f64p]
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, name: str = "") -> CSR:
    """Symmetrise, drop self-loops and duplicates, sort rows."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = src.shape[0]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    bound = ctypes.c_int64(0)
    lib.wlgen_csr_count(n, m, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                        _p(row_ptr, ctypes.c_int64), ctypes.byref(bound))
    col = np.empty(max(bound.value, 1), dtype=np.int32)
    nnz = ctypes.c_int64(0)
    rc = lib.wlgen_csr_fill(n, m, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                            _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32),
                            ctypes.byref(nnz))
    if rc != 0:
        raise MemoryError("csr_fill failed")
    col = col[: nnz.value].copy()
    return CSR(n, row_ptr, col, name)


def csr_from_dense(A: np.ndarray, name: str = "") -> CSR:
    """CSR of a dense symmetric 0/1 matrix (small fixtures)."""
    A = np.asarray(A)
    iu, ju = np.nonzero(np.triu(A, 1))
    return csr_from_edges(A.shape[0], iu, ju, name)


# ---------------------------------------------------------------- small graphs
def g58() -> CSR:
    """Toy network G_{5,8} of Sec. 5.1: path 1-2-3-4-5 plus leaves 6..13 on
    node 3 (edge list of the paper's TikZ drawing, 1-based there)."""
    edges = [(1, 2), (2, 3), (3, 4), (4, 5)] + [(3, j) for j in range(6, 14)]
    e = np.array(edges, dtype=np.int32) - 1
    return csr_from_edges(13, e[:, 0], e[:, 1], "G_{5,8}")


def cycle(n: int) -> CSR:
    i = np.arange(n, dtype=np.int32)
    return csr_from_edges(n, i, (i + 1) % n, f"C_{n}")


def complete(n: int) -> CSR:
    iu, ju = np.triu_indices(n, 1)
    return csr_from_edges(n, iu, ju, f"K_{n}")


def path(n: int) -> CSR:
    i = np.arange(n - 1, dtype=np.int32)
    return csr_from_edges(n, i, i + 1, f"P_{n}")


def star(leaves: int) -> CSR:
    j = np.arange(1, leaves + 1, dtype=np.int32)
    return csr_from_edges(leaves + 1, np.zeros_like(j), j, f"S_{leaves}")


def hypercube(dim: int) -> CSR:
    n = 1 << dim
    src, dst = [], []
    for b in range(dim):
        i = np.arange(n)
        j = i ^ (1 << b)
        keep = i < j
        src.append(i[keep]); dst.append(j[keep])
    return csr_from_edges(n, np.concatenate(src), np.concatenate(dst), f"Q_{dim}")


def torus2d(r: int, c: int) -> CSR:
    """r x c periodic grid (4-regular for r, c >= 3)."""
    idx = np.arange(r * c).reshape(r, c)
    src = np.concatenate([idx.ravel(), idx.ravel()])
    dst = np.concatenate([np.roll(idx, -1, 1).ravel(), np.roll(idx, -1, 0).ravel()])
    return csr_from_edges(r * c, src, dst, f"T_{r}x{c}")


def grid2d(r: int, c: int) -> CSR:
    """r x c 4-neighbour grid (non-periodic)."""
    idx = np.arange(r * c).reshape(r, c)
    h = (idx[:, :-1].ravel(), idx[:, 1:].ravel())
    v = (idx[:-1, :].ravel(), idx[1:, :].ravel())
    return csr_from_edges(r * c, np.concatenate([h[0], v[0]]),
                          np.concatenate([h[1], v[1]]), f"grid_{r}x{c}")


def erdos_renyi(n: int, mean_degree: float, seed: int) -> CSR:
    """G(n, p) with p = mean_degree / (n - 1), sampled by geometric skipping
    over the n(n-1)/2 unordered pairs (Batagelj and Brandes 2005)."""
    rng = np.random.default_rng(seed)
    p = mean_degree / max(n - 1, 1)
    N = n * (n - 1) // 2
    if N == 0 or p <= 0:
        return CSR(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), f"ER_{n}")
    out = []
    pos = -1
    chunk = int(N * p * 1.2) + 1024
    while True:
        gaps = rng.geometric(p, size=chunk)
        lin = pos + np.cumsum(gaps)
        keep = lin < N
        out.append(lin[keep])
        if not keep.all():
            break
        pos = int(lin[-1])
    lin = np.concatenate(out)
    # unrank linear index of the strict upper triangle, row-major
    # row i holds pairs (i, i+1..n-1); offset(i) = i*n - i*(i+1)/2
    i = (n - 2 - np.floor(np.sqrt(-8.0 * lin + 4.0 * n * (n - 1) - 7) / 2.0 - 0.5)).astype(np.int64)
    off = i * n - i * (i + 1) // 2
    j = lin - off + i + 1
    # guard against floating rounding in the unranking
    bad = (j <= i) | (j >= n)
    while bad.any():
        i[bad & (j <= i)] -= 1
        i[bad & (j >= n)] += 1
        off = i * n - i * (i + 1) // 2
        j = lin - off + i + 1
        bad = (j <= i) | (j >= n)
    return csr_from_edges(n, i.astype(np.int32), j.astype(np.int32), f"ER_{n}")


def barabasi_albert(n: int, m: int, seed: int) -> CSR:
    """Preferential attachment (Barabasi and Albert 1999): start from a star on
    m+1 nodes; each new node attaches to m distinct targets drawn with
    probability proportional to degree (repeated-endpoint list method)."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    src = list(range(1, m0))
    dst = [0] * (m0 - 1)
    rep = src + dst  # endpoint list: node appears once per incident edge
    rep_arr = np.empty(2 * n * m + 2 * m0, dtype=np.int64)
    rep_arr[: len(rep)] = rep
    L = len(rep)
    S = []
    D = []
    for v in range(m0, n):
        targets = set()
        while len(targets) < m:
            draws = rng.integers(0, L, size=2 * m)
            for t in rep_arr[draws]:
                targets.add(int(t))
                if len(targets) == m:
                    break
        for t in targets:
            S.append(v); D.append(t)
            rep_arr[L] = v; rep_arr[L + 1] = t
            L += 2
    src = np.array(src + S, dtype=np.int32)
    dst = np.array(dst + D, dtype=np.int32)
    return csr_from_edges(n, src, dst, f"BA_{n}_{m}")


# ---------------------------------------------------------------- large graphs
def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1) -> CSR:
    """R-MAT graph (Chakrabarti et al. 2004), Graph500-style: 2^scale nodes,
    edge_factor * 2^scale generated edges, seeded vertex relabelling,
    symmetrised, duplicates and self-loops removed."""
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.wlgen_rmat_edges(scale, m, a, b, c, seed, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32))
    perm = np.empty(n, dtype=np.int32)
    lib.wlgen_permutation(n, seed, _p(perm, ctypes.c_int32))
    lib.wlgen_relabel(m, _p(perm, ctypes.c_int32), _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32))
    g = csr_from_edges(n, src, dst, f"RMAT_{scale}")
    return g


def uniform(count: int, seed: int, stream: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.float64)
    lib.wlgen_uniform(count, seed, stream, _p(out, ctypes.c_double))
    return out


def chung_lu(n: int, gamma: float = 2.5, mean_degree: float = 12.0,
             seed: int = 1) -> CSR:
    """Chung-Lu power-law graph with minimum degree 1.

    Weights w_i = x_min * U_i^(-1/(gamma-1)), capped at sqrt(n * mean_degree),
    with x_min calibrated (bisection) so that mean(w) = mean_degree; edges
    (i, j) appear independently with probability min(1, w_i w_j / sum(w))
    (Chung and Lu 2002). Every node left isolated is then joined to one
    partner drawn with probability proportional to w, so the minimum degree
    is 1 as the workload asks.
    """
    lib = _load()
    U = uniform(n, seed, 1)
    U = np.maximum(U, 1e-300)
    base = U ** (-1.0 / (gamma - 1.0))
    cap = np.sqrt(n * mean_degree)
    lo, hi = 1e-3, mean_degree
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.minimum(mid * base, cap).mean() < mean_degree:
            lo = mid
        else:
            hi = mid
    w = np.minimum(hi * base, cap)
    order = np.argsort(-w, kind="stable").astype(np.int32)
    capm = int(w.sum() * 0.75 + 10 * np.sqrt(w.sum()) + 1024)
    src = np.empty(capm, dtype=np.int32)
    dst = np.empty(capm, dtype=np.int32)
    m = ctypes.c_int64(0)
    rc = lib.wlgen_chung_lu_edges(n, _p(w, ctypes.c_double), _p(order, ctypes.c_int32), seed, capm,
                                  _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32), ctypes.byref(m))
    if rc == -3:
        capm = int(m.value) + 1024
        src = np.empty(capm, dtype=np.int32)
        dst = np.empty(capm, dtype=np.int32)
        rc = lib.wlgen_chung_lu_edges(n, _p(w, ctypes.c_double), _p(order, ctypes.c_int32), seed,
                                      capm, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                      ctypes.byref(m))
    if rc != 0:
        raise RuntimeError(f"chung_lu generator failed ({rc})")
    src, dst = src[: m.value], dst[: m.value]
    deg = np.bincount(np.concatenate([src, dst]), minlength=n)
    iso = np.nonzero(deg == 0)[0]
    if iso.size:
        cdf = np.cumsum(w) / w.sum()
        r = uniform(iso.size, seed, 2)
        partner = np.searchsorted(cdf, r, side="right").clip(0, n - 1)
        same = partner == iso
        partner[same] = (partner[same] + 1) % n
        src = np.concatenate([src, iso.astype(np.int32)])
        dst = np.concatenate([dst, partner.astype(np.int32)])
    return csr_from_edges(n, src, dst, f"ChungLu_{n}")


# ---------------------------------------------------------------- vectors
def gaussian_block(n: int, k: int, seed: int) -> np.ndarray:
    """n x k standard normal block, row-major float64."""
    return np.random.default_rng(seed).standard_normal((n, k))


def point_sources(g: CSR, k: int, seed: int) -> np.ndarray:
    """k distinct nodes with degree >= 1 drawn uniformly (seeded); returns
    their indices. The block U0 = [e_j1 ... e_jk] is built by the caller."""
    cand = np.nonzero(g.degrees >= 1)[0]
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(cand, size=k, replace=False))


def unit_block(n: int, nodes: np.ndarray) -> np.ndarray:
    U = np.zeros((n, len(nodes)))
    U[nodes, np.arange(len(nodes))] = 1.0
    return U


def batch_graphs(count: int = 64, lo: float = 1e3, hi: float = 2e5, seed: int = 1):
    """Graphs of uneven size for the batched workload: sizes log-uniform in
    [lo, hi], generators cycling Erdos-Renyi (mean degree 10), Barabasi-Albert
    (m = 3) and 2D 4-neighbour grids with r * c ~ size."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    out = []
    for i, s in enumerate(sizes):
        kind = i % 3
        if kind == 0:
            out.append(erdos_renyi(int(s), 10.0, seed * 1000 + i))
        elif kind == 1:
            out.append(barabasi_albert(int(s), 3, seed * 1000 + i))
        else:
            r = max(2, int(round(np.sqrt(s))))
            c = max(2, int(round(s / r)))
            out.append(grid2d(r, c))
    return out
