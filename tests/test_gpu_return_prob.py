"""Average return probability tr(exp(-t L)) / n and its XNysTrace estimate
(Sec. 4.4, Alg. 1) through the C ABI.

Against the oracle's Alg. 1 with exact Y(t) = exp(-t L) Omega and the same
bit-exact Omega: in the FP64 and refined forms the GPU's Y(t) carries only
the Lanczos error (outer_tol) and enters an FP64 Gram, so the estimates
agree within 1e-10 (FP64) / 1e-8 (refined) relative; in the sketch form
Y(t) is rounded to FP32 for the tensor-core Gram (1e-5 relative, as for
wl_trace). Against the exact p(t): within a few error estimates."""
import numpy as np
import pytest

import wlgen
from oracle import graph, philox, walks, xnys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def WL(g, **kw):
    from paper_2601_11338_gb300.api import WalkLaplacian
    return WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, **kw)


ETOL = {"fp64": (1e-10, 1e-6), "refined": (1e-8, 1e-6), "sketch": (1e-5, 1e-2)}


@pytest.mark.parametrize("variant,mu,prec,M,reorder", [("allwalk", 0.0, "fp64", 16, 1), ("nbt", 1.0, "refined", 7, 0),
                                                        ("btdw", 0.5, "refined", 32, 1), ("nbt", 1.0, "sketch", 16, 1),
                                                        ("nbt", 1.0, "sketch_tc", 16, 1)])
def test_estimates_match_oracle_alg1(variant, mu, prec, M, reorder):
    gram = 1 if prec == "sketch_tc" else 0  # sketch_tc: the tensor-core Gram
    prec = "sketch" if gram else prec
    g = wlgen.erdos_renyi(500, 8, 51)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    w = WL(g, variant=variant, mu=mu, alpha_rel=0.5, prec=prec, tol=1e-12, outer_tol=1e-11, reorder=reorder,
           gram=gram)
    L = walks.walk_laplacian(walks.phi_resolvent_closed(A, mu, w.info["alpha"]))
    ts = [0.0, 0.3, 1.0, 2.5]
    seed = 9001 + M
    p, e = w.return_prob(M, seed, ts)
    Om, _ = philox.gaussian_sketch(g.n, M, seed)
    want = xnys.xnys_return_probability(L, Om, ts)
    exact = xnys.return_probability(L, ts)
    for i, (pe, ee) in enumerate(want):
        assert abs(p[i] - pe) <= ETOL[prec][0] * abs(pe), (ts[i], p[i], pe)
        assert abs(e[i] - ee) <= ETOL[prec][1] * ee + 1e-12, (ts[i], e[i], ee)
        assert abs(p[i] - exact[i]) <= 8 * e[i] + 1e-12, (ts[i], p[i], exact[i], e[i])
    w.close()


def test_many_time_points_and_identity_function():
    """Combinatorial Laplacian (identity f) on a cycle: 90 time points in
    [0, 5] (several batches of the combination); the estimates follow the
    Bessel closed form e^{-2t} I_0(2t) of tr(exp(-t L)) / n within their error
    estimates, and decrease from 1."""
    from scipy.special import iv
    n = 600
    g = wlgen.cycle(n)
    w = WL(g, f="identity", outer_tol=1e-11)
    ts = np.linspace(0.0, 5.0, 90)
    p, e = w.return_prob(24, 77, ts)
    exact = np.exp(-2 * ts) * iv(0, 2 * ts)
    assert np.all(np.abs(p - exact) <= 8 * e + 1e-12)
    assert abs(p[0] - 1.0) < 0.05 and p[-1] < p[0]
    w.close()


def test_btdw_exponential_mu_sweep():
    """L_mu(exp) on a 20 x 30 grid for mu in {0, .25, .5, .75, 1} at the
    same beta = 1 / lambda_max(A) and the same Omega: each estimate matches
    the oracle's Alg. 1 (1e-5 relative), and, as in Sec. 4.4's figure on
    varying mu, both the exact values and the estimates rise with mu at every
    t (the common Omega correlates the estimates)."""
    from oracle import spectral
    g = wlgen.grid2d(20, 30)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    beta = 1.0 / spectral.lambda_max(A)
    ts = [0.5, 1.0, 2.0, 4.0]
    M, seed = 32, 4242
    Om, _ = philox.gaussian_sketch(g.n, M, seed)
    got, exact = [], []
    for mu in (0.0, 0.25, 0.5, 0.75, 1.0):
        w = WL(g, variant="btdw", f="exp", beta=beta, mu=mu, prec="refined", tol=1e-12, outer_tol=1e-11)
        p, e = w.return_prob(M, seed, ts)
        w.close()
        L = walks.walk_laplacian(walks.phi_series(A, mu, walks.exp_coeffs(beta)))
        want = xnys.xnys_return_probability(L, Om, ts)
        for i, (pe, ee) in enumerate(want):
            assert abs(p[i] - pe) <= 1e-5 * abs(pe), (mu, ts[i], p[i], pe)
            assert abs(e[i] - ee) <= 1e-2 * ee + 1e-12, (mu, ts[i], e[i], ee)
        got.append(p)
        exact.append(xnys.return_probability(L, ts))
    assert np.all(np.diff(np.array(exact), axis=0) > 0)
    assert np.all(np.diff(np.array(got), axis=0) > 0)


def test_argument_checks():
    from paper_2601_11338_gb300 import wl
    g = wlgen.erdos_renyi(50, 4, 3)
    w = WL(g, alpha_rel=0.5)
    for M, ts in ((1, [0.5]), (65, [0.5]), (8, [-1.0]), (8, [])):
        with pytest.raises(wl.WLError):
            w.return_prob(M, 1, ts)
    w.close()


def test_graph_without_edges():
    """L = 0: exp(-t L) = I at every t, so the estimate is XNysTrace of the
    identity (unbiased for n; its spread is the error estimate)."""
    from paper_2601_11338_gb300.api import WalkLaplacian
    n = 2000
    w = WalkLaplacian(np.zeros(n + 1, np.int32), np.zeros(0, np.int32), n, alpha=0.3)
    p, e = w.return_prob(16, 3, [0.0, 1.0, 50.0])
    assert np.all(np.abs(p - 1.0) <= 6 * e + 1e-12)
    assert abs(p[0] - p[2]) < 1e-12
    w.close()
