"""Shift-and-invert Lanczos for exp(-tau L) u0 and the average return
probability (Sec. 4.4: a rational Krylov space built from solves with the
shifted Laplacian; each shifted solve of the resolvent walk Laplacian is one
CG solve with M - a (D_f + sigma I)^{-1}, followed by one product with M).

The results have the same plain definitions as the polynomial route, so
they are checked against the same oracle: the dense exp(-tau L) by eigh,
the literal leave-one-out XNysTrace of exp(-t L) with the same Omega, and
the spectral closed form of the return probability on a cycle. Tolerances
as in the other parity tests: 1e-10 (FP64 form), 1e-8 (refined form),
norm-wise and element-wise per column."""
import numpy as np
import pytest

import wlgen
from oracle import graph, philox, walks, xnys
from parity_metrics import relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "refined": 1e-8}


def WL(g, **kw):
    from paper_2601_11338_gb300.api import WalkLaplacian
    return WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, **kw)


def oracle_L(g, mu, alpha):
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    return walks.walk_laplacian(walks.phi_resolvent_closed(A, mu, alpha))


@pytest.mark.parametrize("prec", ["fp64", "refined"])
@pytest.mark.parametrize("sigma", [0.3, 3.0])
@pytest.mark.parametrize("variant,mu,reorder", [("allwalk", 0.0, 1), ("nbt", 1.0, 0)])
def test_si_diffusion_matches_oracle(prec, sigma, variant, mu, reorder):
    g = wlgen.erdos_renyi(2000, 8, 20260000)
    w = WL(g, variant=variant, mu=mu, alpha_rel=0.5, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12,
           outer_tol=1e-13, shift=sigma, reorder=reorder)
    L = oracle_L(g, mu, w.info["alpha"])
    nodes = wlgen.point_sources(g, 3, 17)
    U0 = wlgen.unit_block(g.n, nodes)
    taus = [0.1, 1.0, 10.0]
    U = w.expmv(torch.as_tensor(U0, device="cuda"), taus).cpu().numpy()
    st = w.last
    w.close()
    want = walks.diffusion(L, U0, taus)
    for t in range(len(taus)):
        assert relerr(U[t], want[t]) <= TOL[prec], (taus[t], relerr(U[t], want[t]), st.outer_iters)
        np.testing.assert_allclose(U[t].sum(0), 1.0, rtol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_si_near_the_pole_needs_few_steps(prec):
    """alpha = 0.998 / rho(Z_1) on a Chung-Lu graph (n = 4000): the polynomial
    Lanczos run needs hundreds of steps for exp(-10 L) e_hub (the walk degrees
    reach 3.4e3); the shift-and-invert run needs a few dozen."""
    g = wlgen.chung_lu(4000, seed=7)
    w = WL(g, variant="nbt", alpha_rel=0.998, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12,
           outer_tol=1e-12, max_outer=1000, shift=1.0)
    L = oracle_L(g, 1.0, w.info["alpha"])
    hub = int(np.argmax(np.diff(g.row_ptr)))
    U0 = np.zeros((g.n, 1))
    U0[hub, 0] = 1.0
    U = w.expmv(torch.as_tensor(U0, device="cuda"), [10.0]).cpu().numpy()
    steps = w.last.outer_iters
    w.close()
    assert steps <= 100, steps
    want = walks.diffusion(L, U0, [10.0])[0]
    assert relerr(U[0], want) <= TOL[prec], (steps, relerr(U[0], want))
    np.testing.assert_allclose(U[0].sum(0), 1.0, rtol=1e-9)


@pytest.mark.parametrize("prec,etol", [("fp64", 1e-10), ("refined", 1e-8)])
def test_si_return_probability_matches_alg1(prec, etol):
    g = wlgen.erdos_renyi(500, 8, 51)
    w = WL(g, variant="nbt", alpha_rel=0.5, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12, outer_tol=1e-12,
           shift=0.5)
    L = oracle_L(g, 1.0, w.info["alpha"])
    ts = [0.0, 0.3, 1.0, 2.5, 20.0]
    M, seed = 16, 4242
    p, e = w.return_prob(M, seed, ts)
    w.close()
    Om, _ = philox.gaussian_sketch(g.n, M, seed)
    want = xnys.xnys_return_probability(L, Om, ts)
    exact = xnys.return_probability(L, ts)
    for i, (pe, ee) in enumerate(want):
        assert abs(p[i] - pe) <= etol * abs(pe), (ts[i], p[i], pe)
        assert abs(e[i] - ee) <= 1e-6 * ee + 1e-12, (ts[i], e[i], ee)
        assert abs(p[i] - exact[i]) <= 8 * e[i] + 1e-12, (ts[i], p[i], exact[i], e[i])


def test_si_return_probability_with_a_padded_column_block():
    """M = 7 test vectors run as a block of 8 columns, one of them zero: the
    run stops by the rule (the zero column's y stays zero) instead of running
    to its step cap, and the estimates match Alg. 1 with the oracle's Y."""
    g = wlgen.erdos_renyi(500, 8, 51)
    w = WL(g, variant="nbt", alpha_rel=0.5, prec="refined", tol=1e-12, outer_tol=1e-10, shift=0.5, max_outer=150)
    L = oracle_L(g, 1.0, w.info["alpha"])
    ts = [0.0, 0.3, 1.0, 2.5, 20.0]
    M, seed = 7, 4243
    p, e = w.return_prob(M, seed, ts)
    steps, status = w.last.outer_iters, w.last.status
    w.close()
    assert status == 0 and steps < 150, (status, steps)
    Om, _ = philox.gaussian_sketch(g.n, M, seed)
    want = xnys.xnys_return_probability(L, Om, ts)
    for i, (pe, ee) in enumerate(want):
        assert abs(p[i] - pe) <= 1e-8 * abs(pe), (ts[i], p[i], pe)
        assert abs(e[i] - ee) <= 1e-6 * ee + 1e-12, (ts[i], e[i], ee)


def test_si_return_probability_on_a_cycle_closed_form():
    """C_n is 2-regular, so M = (a + alpha^2 mu 2) I - alpha A shares A's
    eigenvectors and L has eigenvalues g(2) - g(2 cos(2 pi j / n)) with
    g(lam) = a / (a + 2 alpha^2 mu - alpha lam): tr(exp(-t L)) / n is a sum of
    exponentials. The estimate (M = 32, a long time range in one run) lies
    within a few error estimates of it."""
    n = 3000
    g = wlgen.cycle(n)
    mu = 1.0
    w = WL(g, variant="nbt", alpha_rel=0.5, prec="refined", tol=1e-12, outer_tol=1e-10, shift=0.05)
    alpha = w.info["alpha"]
    ts = np.concatenate([[0.0], np.geomspace(0.1, 1000.0, 40)])
    p, e = w.return_prob(32, 99, ts)
    steps = w.last.outer_iters
    w.close()
    a = 1.0 - mu * mu * alpha * alpha
    gfun = lambda lam: a / (a + 2 * alpha * alpha * mu - alpha * lam)
    lam = gfun(2.0) - gfun(2.0 * np.cos(2 * np.pi * np.arange(n) / n))
    exact = np.array([np.exp(-t * lam).mean() for t in ts])
    assert np.all(np.abs(p - exact) <= 8 * e + 1e-10), np.abs(p - exact) / np.maximum(e, 1e-300)
    assert abs(p[0] - 1.0) < 0.05
    assert steps < 200, steps


def test_si_needs_the_resolvent():
    from paper_2601_11338_gb300 import wl
    g = wlgen.cycle(50)
    w = WL(g, f="identity", shift=1.0)
    U0 = torch.zeros((g.n, 1), dtype=torch.float64, device="cuda")
    U0[0, 0] = 1.0
    w.expmv(U0, [1.0], allow=(wl.WL_ERR_UNSUPPORTED,))
    assert w.last.status == wl.WL_ERR_UNSUPPORTED
    w.close()


@pytest.mark.parametrize("prec", ["fp64", "refined"])
def test_si_with_reorthogonalisation(prec):
    """The shift-and-invert basis kept orthogonal (reorth = 1) gives the same
    diffusion within the tolerances, in no more steps."""
    g = wlgen.barabasi_albert(1500, 3, 21)
    L = oracle_L(g, 1.0, WL(g, variant="nbt", alpha_rel=0.9).info["alpha"])
    U0 = wlgen.unit_block(g.n, wlgen.point_sources(g, 2, 3))
    steps = {}
    for reorth in (0, 1):
        w = WL(g, variant="nbt", alpha_rel=0.9, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12, outer_tol=1e-12,
               shift=1.0, reorth=reorth)
        U = w.expmv(torch.as_tensor(U0, device="cuda"), [0.5, 5.0]).cpu().numpy()
        steps[reorth] = w.last.outer_iters
        assert w.last.reorth_blocks == (steps[reorth] - 1 if reorth else 0)
        w.close()
        want = walks.diffusion(L, U0, [0.5, 5.0])
        for t in range(2):
            assert relerr(U[t], want[t]) <= TOL[prec], (reorth, t, relerr(U[t], want[t]))
    assert steps[1] <= steps[0], steps
