"""Batched executor (many graphs x many mu values in one CUDA graph launch)
against the CPU FP64 oracle, problem by problem.

Tolerances as for the single-graph path: relative 2-norm and largest element-wise error (relative to the column's largest entry) per output column,
1e-10 for the FP64 form and 1e-8 for the refined form.
"""
import numpy as np
import pytest

import wlgen
from oracle import graph, spectral, walks
from parity_metrics import relerr  # max of norm-wise and element-wise error per column

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "refined": 1e-8}
MUS = [1.0, 0.75, 0.5, 0.25, 0.0]  # theta = 1 - mu in {0, .25, .5, .75, 1}


def small_graphs():
    # sizes and structure of the batched workload, scaled down so that the
    # dense oracle runs in seconds; the star has a row of 300 entries and
    # exercises the one-CTA-per-row hub tiles
    return [
        wlgen.erdos_renyi(300, 10.0, 11),
        wlgen.barabasi_albert(400, 3, 12),
        wlgen.grid2d(15, 20),
        wlgen.star(300),
        wlgen.erdos_renyi(517, 6.0, 13),
        wlgen.path(37),
    ]


def build(gs, prec, tol, **kw):
    from paper_2601_11338_gb300 import wl
    p = wl.make_params(f=wl.WL_F_RESOLVENT, alpha_rel=0.5, prec=wl.WL_REFINED if prec == "refined" else wl.WL_FP64,
                       tol=tol, max_iter=kw.get("max_iter", 0), stream=torch.cuda.current_stream().cuda_stream)
    graphs = [(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz) for g in gs]
    return wl.wl_batch_build(graphs, kw.get("mus", MUS), p)


def run(b, gs, V, k, stepped=0, allow=()):
    from paper_2601_11338_gb300 import wl
    n = sum(g.n for g in gs)
    nmu = b.nmu
    Df = torch.empty((nmu, n), dtype=torch.float64, device="cuda")
    W = torch.empty((nmu, n, k), dtype=torch.float64, device="cuda")
    st = wl.wl_stats()
    rc = wl.wl_batch_run(b, V, k, Df, W, stepped, st, allow)
    torch.cuda.synchronize()
    return Df.cpu().numpy(), W.cpu().numpy(), st, rc


@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_batch_matches_oracle_per_problem(prec):
    from paper_2601_11338_gb300 import wl
    gs = small_graphs()
    k = 4
    n = sum(g.n for g in gs)
    Vh = wlgen.gaussian_block(n, k, 5)
    # stopping rule of the solves (the parity bar is TOL): the refined form
    # tests the true residual, whose floor is about u64 |M| |x| / |b| ~ 1e-12
    # on the star at mu = 1 (kappa(M) ~ 8e3 at alpha = 0.5 / rho(Z_1) = 0.5)
    b = build(gs, prec, 1e-13 if prec == "fp64" else 1e-11)
    Df, W, st, rc = run(b, gs, torch.as_tensor(Vh, device="cuda"), k)
    assert rc == wl.WL_OK and st.launches == 1
    off = np.concatenate([[0], np.cumsum([g.n for g in gs])])
    for gi, g in enumerate(gs):
        A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
        lmax = spectral.lambda_max(A)
        for j, mu in enumerate(MUS):
            info = wl.wl_batch_info(b, gi, j)
            rho = spectral.rho_companion(A, mu) if mu > 0 else lmax
            assert abs(info["rho"] - rho) <= 1e-8 * rho, (gi, mu)
            assert abs(info["lambda_max"] - lmax) <= 1e-9 * lmax
            alpha = info["alpha"]
            assert abs(alpha * info["rho"] - 0.5) <= 1e-12
            phi = walks.phi_resolvent_closed(A, mu, alpha)
            sl = slice(off[gi], off[gi + 1])
            assert relerr(Df[j, sl], walks.walk_degrees(phi)) <= TOL[prec], (gi, mu)
            assert relerr(W[j, sl], walks.apply_laplacian(phi, Vh[sl])) <= TOL[prec], (gi, mu)
    b.destroy()


@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_batch_graph_equals_stepped_and_replays(prec):
    """One CUDA graph launch gives bit for bit the result of the same kernels
    launched one by one, and replaying the graph repeats it exactly."""
    gs = small_graphs()
    k = 8
    n = sum(g.n for g in gs)
    V = torch.as_tensor(wlgen.gaussian_block(n, k, 6), device="cuda")
    b = build(gs, prec, 1e-12 if prec == "fp64" else 1e-10)
    D1, W1, s1, _ = run(b, gs, V, k, stepped=0)
    D2, W2, s2, _ = run(b, gs, V, k, stepped=1)
    D3, W3, s3, _ = run(b, gs, V, k, stepped=0)
    assert s1.launches == 1 and s2.launches == 0
    assert np.array_equal(D1, D2) and np.array_equal(W1, W2)
    assert np.array_equal(D1, D3) and np.array_equal(W1, W3)
    b.destroy()


def test_batch_host_buffers_and_ones_in_kernel():
    """Host arrays in and out; L 1 = 0 for every problem (rows of the walk
    Laplacian sum to zero), D_f > 0."""
    from paper_2601_11338_gb300 import wl
    gs = [wlgen.barabasi_albert(2000, 3, 21), wlgen.grid2d(30, 40), wlgen.erdos_renyi(3000, 10.0, 22)]
    n = sum(g.n for g in gs)
    b = build(gs, "refined", 1e-10)
    V = np.ones((n, 1))
    Df = np.empty((len(MUS), n))
    W = np.empty((len(MUS), n, 1))
    st = wl.wl_stats()
    assert wl.wl_batch_run(b, V, 1, Df, W, 0, st) == wl.WL_OK
    assert (Df > 0).all()
    assert np.abs(W).max() <= 1e-8 * np.abs(Df).max()
    b.destroy()


def test_batch_iteration_cap_reports_no_convergence():
    from paper_2601_11338_gb300 import wl
    gs = small_graphs()[:3]
    n = sum(g.n for g in gs)
    b = build(gs, "fp64", 1e-14, max_iter=3)
    V = torch.as_tensor(wlgen.gaussian_block(n, 2, 7), device="cuda")
    _, _, st, rc = run(b, gs, V, 2, allow=(wl.WL_ERR_NO_CONVERGENCE,))
    assert rc == wl.WL_ERR_NO_CONVERGENCE
    info = wl.wl_batch_info(b, 0, 0)
    assert info["iters_v"] == 3 and info["status"] == wl.WL_ERR_NO_CONVERGENCE
    b.destroy()


def test_batch_rejects_bad_input():
    from paper_2601_11338_gb300 import wl
    g = wlgen.cycle(10)
    bad_rp = g.row_ptr.astype(np.int32).copy()
    col = g.col_idx.copy()
    col[0], col[1] = col[1], col[0]  # unsorted row
    p = wl.make_params(f=wl.WL_F_RESOLVENT, alpha_rel=0.5)
    with pytest.raises(wl.WLError):
        wl.wl_batch_build([(bad_rp, col, g.n, g.nnz)], [1.0], p)
    with pytest.raises(wl.WLError):
        wl.wl_batch_build([(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz)], [1.5], p)
    p2 = wl.make_params(f=wl.WL_F_RESOLVENT, alpha=0.6)  # alpha * rho(C_10) = 1.2
    with pytest.raises(wl.WLError):
        wl.wl_batch_build([(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz)], [0.0], p2)


def test_batch_workload_sampled_against_single_graph_path():
    """A 16-graph slice of the batched workload (sizes log-uniform in
    [1e3, 2e4], ER / BA / grid), k = 32: a few problems are checked against
    the single-graph path (itself parity-tested against the oracle)."""
    from paper_2601_11338_gb300 import wl
    from paper_2601_11338_gb300.api import WalkLaplacian
    gs = wlgen.batch_graphs(16, 1e3, 2e4, seed=3)
    k = 32
    n = sum(g.n for g in gs)
    Vh = wlgen.gaussian_block(n, k, 8)
    V = torch.as_tensor(Vh, device="cuda")
    b = build(gs, "refined", 1e-10)
    Df, W, st, rc = run(b, gs, V, k)
    assert rc == wl.WL_OK
    assert wl.wl_batch_tile_rows(b, k) in (64, 128, 256, 512)
    off = np.concatenate([[0], np.cumsum([g.n for g in gs])])
    for gi, j in [(0, 0), (1, 1), (2, 4), (7, 2), (13, 3)]:
        g = gs[gi]
        info = wl.wl_batch_info(b, gi, j)
        w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="btdw", mu=MUS[j],
                          alpha=info["alpha"], prec="fp64", tol=1e-13)
        sl = slice(off[gi], off[gi + 1])
        Dref = w.degrees().cpu().numpy()
        Wref = w.apply(V[sl].contiguous()).cpu().numpy()
        assert relerr(Df[j, sl], Dref) <= 1e-8, (gi, j)
        assert relerr(W[j, sl], Wref) <= 1e-8, (gi, j)
    b.destroy()


def test_batch_spectral_scales_with_more_graphs_than_search_threads():
    """150 small graphs (more than the build runs searches for at a time, so
    host threads take several graphs each and the mu searches join and leave
    the shared rounds as they go): every lambda_max(A) and rho(Z_mu) against the
    oracle's dense eigenvalues, and the build reports its shared rounds."""
    from paper_2601_11338_gb300 import wl
    rng = np.random.default_rng(17)
    gs = []
    for i in range(150):
        kind = i % 3
        if kind == 0:
            gs.append(wlgen.erdos_renyi(int(rng.integers(20, 80)), 5.0, 100 + i))
        elif kind == 1:
            gs.append(wlgen.barabasi_albert(int(rng.integers(20, 80)), 2, 100 + i))
        else:
            gs.append(wlgen.grid2d(int(rng.integers(3, 9)), int(rng.integers(3, 9))))
    mus = [1.0, 0.5, 0.0]
    p = wl.make_params(f=wl.WL_F_RESOLVENT, alpha_rel=0.5, prec=wl.WL_FP64, tol=1e-12,
                       stream=torch.cuda.current_stream().cuda_stream)
    st = wl.wl_stats()
    b = wl.wl_batch_build([(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz) for g in gs], mus, p, st)
    assert st.status == wl.WL_OK and st.outer_iters > 0
    for gi, g in enumerate(gs):
        A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
        lmax = spectral.lambda_max(A)
        for j, mu in enumerate(mus):
            info = wl.wl_batch_info(b, gi, j)
            assert abs(info["lambda_max"] - lmax) <= 1e-9 * lmax, (gi, mu)
            rho = spectral.rho_companion(A, mu) if mu > 0 else lmax
            assert abs(info["rho"] - rho) <= 1e-8 * rho, (gi, mu)
    b.destroy()


def test_batch_invalid_graph_among_valid_ones_fails_without_hanging():
    """One unsorted graph among 40 valid ones: its search thread fails at
    validation and leaves while the others are in their shared rounds; the
    build reports the error (in bounded time) and the next build works."""
    import time
    from paper_2601_11338_gb300 import wl
    gs = [wlgen.erdos_renyi(200 + 7 * i, 6.0, 300 + i) for i in range(40)]
    graphs = [(g.row_ptr.astype(np.int32), g.col_idx.copy(), g.n, g.nnz) for g in gs]
    col = graphs[17][1]
    col[0], col[1] = col[1], col[0]  # an unsorted row
    p = wl.make_params(f=wl.WL_F_RESOLVENT, alpha_rel=0.5, prec=wl.WL_FP64, tol=1e-12,
                       stream=torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    with pytest.raises(wl.WLError):
        wl.wl_batch_build(graphs, [1.0, 0.5, 0.0], p)
    assert time.perf_counter() - t0 < 60.0
    good = [(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz) for g in gs[:5]]
    b = wl.wl_batch_build(good, [1.0, 0.5, 0.0], p)
    A = graph.dense_adjacency(gs[3].row_ptr, gs[3].col_idx, gs[3].n)
    info = wl.wl_batch_info(b, 3, 0)
    rho = spectral.rho_companion(A, 1.0)
    assert abs(info["rho"] - rho) <= 1e-8 * rho
    b.destroy()
