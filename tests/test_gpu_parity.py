"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (relative 2-norm, and largest element-wise error relative to the
column's largest entry, per output column and per tau):
  FP64 form   1e-10     (inner CG tol 1e-13, Lanczos target 1e-12)
  refined     1e-8      (FP32 inner CG with double-float residual and update)
"""
import numpy as np
import pytest

import wlgen
from oracle import graph, spectral, walks
from parity_metrics import relerr  # max of norm-wise and element-wise error per column

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "refined": 1e-8}


def dense(g):
    return graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)


def WL(g, **kw):
    from paper_2601_11338_gb300.api import WalkLaplacian
    return WalkLaplacian(g.row_ptr[:].astype(np.int32), g.col_idx, g.n, **kw)


def cpu(t):
    return t.detach().cpu().numpy()


def oracle_for(A, mu, alpha):
    phi = walks.phi_resolvent_closed(A, mu, alpha)
    return phi, walks.walk_degrees(phi), walks.walk_laplacian(phi)


# ------------------------------------------------------------ the small workload
@pytest.mark.parametrize("reorder", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_erdos_renyi_allwalk_resolvent(prec, reorder):
    """ER n = 2000, mean degree 8, all-walk resolvent, alpha = 0.5 / lambda_max(A):
    D_f, L V for 4 Gaussian vectors, exp(-tau L) e_1 at tau = 1."""
    g = wlgen.erdos_renyi(2000, 8, 20260000)
    A = dense(g)
    w = WL(g, variant="allwalk", alpha_rel=0.5, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12,
           outer_tol=1e-13, reorder=reorder)
    info = w.info
    lmax = spectral.lambda_max(A)
    assert abs(info["lambda_max"] - lmax) <= 1e-9 * lmax
    assert abs(info["alpha"] * lmax - 0.5) <= 1e-9
    phi, Df, L = oracle_for(A, 0.0, info["alpha"])
    assert relerr(cpu(w.degrees()), Df) <= TOL[prec]
    V = wlgen.gaussian_block(g.n, 4, 20260001)
    W = w.apply(torch.as_tensor(V, device="cuda"))
    assert relerr(cpu(W), L @ V) <= TOL[prec]
    U0 = np.zeros((g.n, 1)); U0[0, 0] = 1.0
    U = w.expmv(torch.as_tensor(U0, device="cuda"), [1.0])
    want = walks.diffusion(L, U0, [1.0])[0]
    assert relerr(cpu(U[0]), want) <= TOL[prec]


# ------------------------------------------------------------ variants, ragged blocks, hubs
def hub_graph():
    """ER graph plus a hub joined to 700 nodes and a mid-degree node (rows in
    every work class of the kernels) and a few isolated nodes."""
    g = wlgen.erdos_renyi(900, 6, 7)
    src = [0] * 700 + [1] * 40
    dst = list(range(100, 800)) + list(range(200, 240))
    rp, ci = g.row_ptr, g.col_idx
    e_src = np.repeat(np.arange(g.n), np.diff(rp))
    keep = e_src < ci
    s = np.concatenate([e_src[keep], src])
    d = np.concatenate([ci[keep], dst])
    n = g.n + 3  # three isolated nodes at the end
    return wlgen.csr_from_edges(n, s, d, "hub")


@pytest.mark.parametrize("reorder", [0, 1, 2])
@pytest.mark.parametrize("variant,mu", [("nbt", 1.0), ("btdw", 0.5), ("btdw", 0.25), ("allwalk", 0.0)])
@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_variants_apply_and_degrees(variant, mu, prec, reorder):
    g = hub_graph()
    A = dense(g)
    w = WL(g, variant=variant, mu=mu, alpha_rel=0.5, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12,
           reorder=reorder)
    info = w.info
    rho = spectral.rho_companion(A, mu)
    assert abs(info["rho"] - rho) <= 1e-7 * rho
    phi, Df, L = oracle_for(A, mu, info["alpha"])
    assert relerr(cpu(w.degrees()), Df) <= TOL[prec]
    for k in (5, 33):  # ragged column blocks: 4 + 1, 32 + 1
        V = wlgen.gaussian_block(g.n, k, 100 + k)
        W = w.apply(torch.as_tensor(V, device="cuda"))
        assert relerr(cpu(W), L @ V) <= TOL[prec], k


@pytest.mark.parametrize("prec,reorth", [("fp64", 1), ("refined", 1), ("refined", 0)])
def test_long_lanczos_run_near_the_pole(prec, reorth):
    """alpha = 0.998 / rho(Z_1) on a Chung-Lu graph (n = 4000): the hub's walk
    degree reaches about 3.4e3, so exp(-10 L) e_hub takes hundreds of Lanczos
    steps (the oracle's own run without reorthogonalisation needs 512): the
    long basis and the block evaluation of exp(-tau T_m) e_1 (more than 128
    steps). With the basis kept orthogonal (reorth = 1) the run is shorter
    and its check-to-check stopping rule bounds the error tightly; the
    refined form is also run on the plain recurrence."""
    g = wlgen.chung_lu(4000, seed=7)
    A = dense(g)
    w = WL(g, variant="nbt", alpha_rel=0.998, prec=prec, tol=1e-14 if prec == "fp64" else 1e-12,
           outer_tol=1e-12, max_outer=1000, reorth=reorth)
    phi, Df, L = oracle_for(A, 1.0, w.info["alpha"])
    hub = int(np.argmax(A.sum(axis=1)))
    U0 = np.zeros((g.n, 1))
    U0[hub, 0] = 1.0
    U = cpu(w.expmv(torch.as_tensor(U0, device="cuda"), [10.0]))
    steps = w.last.outer_iters
    nre = w.last.reorth_blocks
    w.close()
    assert Df.max() > 2e3
    assert steps > 256, steps
    assert nre == (steps - 1 if reorth else 0), (nre, steps)  # every block but the last one's successor
    want = walks.diffusion(L, U0, [10.0])[0]
    assert relerr(U[0], want) <= TOL[prec], (steps, relerr(U[0], want))
    np.testing.assert_allclose(U[0].sum(0), 1.0, rtol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_nbt_diffusion_several_taus(prec):
    g = wlgen.barabasi_albert(700, 3, 11)
    A = dense(g)
    w = WL(g, variant="nbt", alpha_rel=0.5, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12, outer_tol=1e-13)
    phi, Df, L = oracle_for(A, 1.0, w.info["alpha"])
    nodes = wlgen.point_sources(g, 3, 5)
    U0 = wlgen.unit_block(g.n, nodes)
    taus = [0.1, 1.0, 10.0]
    U = cpu(w.expmv(torch.as_tensor(U0, device="cuda"), taus))
    want = walks.diffusion(L, U0, taus)
    for t in range(3):
        assert relerr(U[t], want[t]) <= TOL[prec], taus[t]
        # mass conservation and positivity (Prop. still-again-an-mmatrix)
        np.testing.assert_allclose(U[t].sum(0), 1.0, rtol=1e-9)
        assert U[t].min() >= -1e-12


@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_identity_function_is_combinatorial_laplacian(reorder):
    g = hub_graph()
    A = dense(g)
    L = graph.combinatorial_laplacian(A)
    w = WL(g, f="identity", reorder=reorder)
    np.testing.assert_array_equal(cpu(w.degrees()), A.sum(1))
    V = wlgen.gaussian_block(g.n, 8, 3)
    np.testing.assert_allclose(cpu(w.apply(torch.as_tensor(V, device="cuda"))), L @ V, rtol=0, atol=1e-12)
    U0 = wlgen.unit_block(g.n, np.array([0, 5]))
    U = cpu(w.expmv(torch.as_tensor(U0, device="cuda"), [0.5, 2.0]))
    want = walks.diffusion(L, U0, [0.5, 2.0])
    for t in range(2):
        assert relerr(U[t], want[t]) <= 1e-10


@pytest.mark.parametrize("mu", [0.5, 1.0])
def test_spectral_radius_of_companion(mu):
    g = wlgen.erdos_renyi(300, 7, 2)
    A = dense(g)
    w = WL(g, variant="btdw", mu=mu, alpha_rel=0.5)
    rho = spectral.rho_companion(A, mu)
    assert abs(w.info["rho"] - rho) <= 1e-8 * rho


@pytest.mark.parametrize("n", [12, 3000])
def test_spectral_radius_double_root_on_a_cycle(n):
    """mu = 1 on a cycle: d = 2 and h(lambda) = 2 - 1/lambda - lambda touches
    zero at lambda = 1 without changing sign (a double root), and rho(Z_1) = 1
    (the dense eigenvalues of Z agree)."""
    g = wlgen.cycle(n)
    if n <= 12:
        assert abs(spectral.rho_companion(dense(g), 1.0) - 1.0) <= 1e-6
    w = WL(g, variant="nbt", alpha_rel=0.5)
    assert abs(w.info["rho"] - 1.0) <= 1e-6, w.info["rho"]
    w.close()


# ------------------------------------------------------------ edge cases
def test_graph_without_edges():
    n = 10
    rp = np.zeros(n + 1, dtype=np.int32)
    from paper_2601_11338_gb300.api import WalkLaplacian
    w = WalkLaplacian(rp, np.zeros(0, np.int32), n, alpha=0.3)
    np.testing.assert_allclose(cpu(w.degrees()), np.ones(n), rtol=1e-15)  # c_0 = 1
    V = torch.randn(n, 3, dtype=torch.float64, device="cuda")
    assert cpu(w.apply(V)).max() == 0.0
    U = cpu(w.expmv(V, [1.0]))
    np.testing.assert_allclose(U[0], cpu(V), rtol=1e-14)


def test_zero_columns_and_k_zero():
    g = wlgen.erdos_renyi(300, 6, 4)
    w = WL(g, alpha_rel=0.5)
    V = torch.zeros(g.n, 3, dtype=torch.float64, device="cuda")
    V[5, 1] = 1.0
    W = cpu(w.apply(V))
    assert np.all(W[:, 0] == 0) and np.all(W[:, 2] == 0)
    U = cpu(w.expmv(V, [1.0]))
    assert np.all(U[0][:, 0] == 0) and np.all(U[0][:, 2] == 0)
    from paper_2601_11338_gb300 import wl
    st = wl.wl_stats()
    assert wl.wl_apply(w.h, V, 3, 0, V, 3, st) == 0


def _csr_arrays(edges, n):
    g = wlgen.csr_from_edges(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    return g.row_ptr.astype(np.int32), g.col_idx.copy()


def test_invalid_graphs_are_rejected():
    from paper_2601_11338_gb300 import wl
    from paper_2601_11338_gb300.api import WalkLaplacian
    rp, ci = _csr_arrays([(0, 1), (1, 2), (2, 3)], 4)
    bad = ci.copy(); bad[0] = 2  # row 0 -> 2 without 2 -> 0
    with pytest.raises(wl.WLError) as e:
        WalkLaplacian(rp, bad, 4, alpha=0.1)
    assert e.value.status in (wl.WL_ERR_NOT_SYMMETRIC, wl.WL_ERR_UNSORTED)
    loop = ci.copy(); loop[0] = 0
    with pytest.raises(wl.WLError) as e:
        WalkLaplacian(rp, loop, 4, alpha=0.1)
    assert e.value.status in (wl.WL_ERR_SELF_LOOP, wl.WL_ERR_NOT_SYMMETRIC)
    uns = ci.copy(); uns[1:3] = uns[1:3][::-1]  # row 1 = (2, 0): unsorted
    with pytest.raises(wl.WLError) as e:
        WalkLaplacian(rp, uns, 4, alpha=0.1)
    assert e.value.status == wl.WL_ERR_UNSORTED
    oob = ci.copy(); oob[-1] = 9
    with pytest.raises(wl.WLError) as e:
        WalkLaplacian(rp, oob, 4, alpha=0.1)
    assert e.value.status == wl.WL_ERR_UNSORTED


def test_alpha_out_of_range_is_rejected():
    from paper_2601_11338_gb300 import wl
    g = wlgen.erdos_renyi(200, 6, 1)
    with pytest.raises(wl.WLError) as e:
        WL(g, variant="nbt", alpha_rel=1.2)
    assert e.value.status == wl.WL_ERR_ALPHA_RANGE


def test_iteration_cap_reports_no_convergence():
    from paper_2601_11338_gb300 import wl
    g = wlgen.erdos_renyi(500, 8, 2)
    w = WL(g, alpha_rel=0.9, max_iter=2, tol=1e-14)
    rc = wl.wl_degrees(w.h, torch.empty(g.n, dtype=torch.float64, device="cuda"), w.last,
                       allow=(wl.WL_ERR_NO_CONVERGENCE,))
    assert rc == wl.WL_ERR_NO_CONVERGENCE and w.last.iters == 2


@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_host_pointers_match_device_pointers(reorder):
    g = wlgen.erdos_renyi(800, 8, 9)
    w = WL(g, alpha_rel=0.5, tol=1e-13, reorder=reorder)
    from paper_2601_11338_gb300 import wl
    V = wlgen.gaussian_block(g.n, 4, 1)
    Wh = np.zeros_like(V)
    wl.wl_apply(w.h, V, 4, 4, Wh, 4)
    Wd = cpu(w.apply(torch.as_tensor(V, device="cuda")))
    np.testing.assert_array_equal(Wh, Wd)
    Dh = np.zeros(g.n)
    wl.wl_degrees(w.h, Dh)
    np.testing.assert_array_equal(Dh, cpu(w.degrees()))


def test_reruns_are_bit_identical():
    g = hub_graph()
    w = WL(g, variant="nbt", alpha_rel=0.5, prec="refined", tol=1e-10)
    V = torch.as_tensor(wlgen.gaussian_block(g.n, 16, 2), device="cuda")
    a = cpu(w.apply(V))
    b = cpu(w.apply(V))
    np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------ full size: properties and closed forms
@pytest.mark.parametrize("reorder", [1, 2])
def test_torus_closed_form_large(reorder):
    """4-regular torus 600 x 500 (n = 3e5): D_f and exp(-tau L) e_1 against the
    closed forms of a d-regular graph (eigenvalues of A are
    2 cos(2 pi j / r) + 2 cos(2 pi k / c)); degree relabelling and reverse
    Cuthill-McKee relabelling inside the handle."""
    r, c, d, mu = 600, 500, 4, 1.0
    g = wlgen.torus2d(r, c)
    w = WL(g, variant="nbt", alpha_rel=0.5, tol=1e-13, outer_tol=1e-12, reorder=reorder)
    info = w.info
    assert abs(info["rho"] - (d - mu)) <= 1e-8 * (d - mu)
    alpha = info["alpha"]
    a = 1 - mu * mu * alpha * alpha
    Df = cpu(w.degrees())
    np.testing.assert_allclose(Df, a / (a + alpha ** 2 * mu * d - alpha * d), rtol=1e-11)
    f = lambda lam: a / (a + alpha ** 2 * mu * d - alpha * lam)
    jj = np.arange(r)[:, None]
    kk = np.arange(c)[None, :]
    lam = 2 * np.cos(2 * np.pi * jj / r) + 2 * np.cos(2 * np.pi * kk / c)
    tau = 2.0
    spec = np.exp(-tau * (f(d) - f(lam)))
    want = np.real(np.fft.ifft2(spec)).ravel()  # circulant: u = F^{-1} (exp(-tau ev)) for e_0
    U0 = torch.zeros(g.n, 1, dtype=torch.float64, device="cuda")
    U0[0, 0] = 1.0
    U = cpu(w.expmv(U0, [tau]))[0][:, 0]
    assert relerr(U, want) <= 1e-10


def test_chung_lu_million_properties():
    """The benchmark graph (Chung-Lu, n = 1e6, NBT): residuals of sampled rows
    recomputed on the CPU in FP64, L 1 = 0, mass conservation, positivity."""
    g = wlgen.chung_lu(1_000_000, seed=20260100)
    w = WL(g, variant="nbt", alpha_rel=0.5, prec="refined", tol=1e-11, outer_tol=1e-10)
    info = w.info
    alpha, mu = info["alpha"], 1.0
    a = 1 - alpha * alpha
    Df = cpu(w.degrees())
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.choice(g.n, 200, replace=False), [int(np.argmax(g.degrees))]])
    for i in rows:
        nb = g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]]
        res = a * Df[i] - alpha * Df[nb].sum() + alpha * alpha * mu * len(nb) * Df[i] - a
        assert abs(res) <= 1e-9 * max(1.0, Df.max()), i
    ones = torch.ones(g.n, 2, dtype=torch.float64, device="cuda")
    Lones = cpu(w.apply(ones))
    assert np.abs(Lones).max() <= 1e-8 * Df.max()
    nodes = wlgen.point_sources(g, 16, 20260101)
    U0 = torch.as_tensor(wlgen.unit_block(g.n, nodes), device="cuda")
    U = cpu(w.expmv(U0, [0.1, 1.0, 10.0]))
    for t in range(3):
        np.testing.assert_allclose(U[t].sum(0), 1.0, rtol=1e-8)
        assert U[t].min() >= -1e-9
