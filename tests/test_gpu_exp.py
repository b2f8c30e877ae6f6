"""The exponential walk function f(x) = exp(beta x) (Def. BDTW-Laplacian with
c_k = beta^k / k!) for mu in [0, 1]: walk degrees, Laplacian action,
diffusion and the discrete-time chain through the C ABI, against the CPU FP64
oracle's series (and, for mu = 0, the spectral form exp(beta A)).

The series runs in double-float arithmetic in both precision forms;
tolerance 1e-10 relative per column.
"""
import numpy as np
import pytest

import wlgen
from oracle import graph, spectral, walks
from parity_metrics import relerr  # max of norm-wise and element-wise error per column

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def dense(g):
    return graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)


def WL(g, **kw):
    from paper_2601_11338_gb300.api import WalkLaplacian
    return WalkLaplacian(g.row_ptr[:].astype(np.int32), g.col_idx, g.n, f="exp", **kw)


@pytest.mark.parametrize("variant,mu", [("allwalk", 0.0), ("btdw", 0.5), ("nbt", 1.0)])
@pytest.mark.parametrize("beta", [0.0, 0.35])
@pytest.mark.parametrize("prec,reorder", [("fp64", 1), ("refined", 0)])
def test_exp_degrees_apply_diffusion(variant, mu, beta, prec, reorder):
    g = wlgen.erdos_renyi(300, 6, 41)
    A = dense(g)
    w = WL(g, variant=variant, mu=mu, beta=beta, prec=prec, tol=1e-13, outer_tol=1e-12, reorder=reorder)
    b = w.info["beta"]
    want_b = beta if beta > 0 else 1.0 / spectral.lambda_max(A)
    assert abs(b - want_b) <= 1e-9 * want_b
    phi = walks.phi_series(A, mu, walks.exp_coeffs(b))
    if mu == 0.0:  # two independent forms agree
        np.testing.assert_allclose(phi, walks.phi_allwalk_exp_eig(A, b), rtol=0, atol=1e-12 * np.abs(phi).max())
    Df = w.degrees().cpu().numpy()
    assert relerr(Df, walks.walk_degrees(phi)) <= TOL
    V = wlgen.gaussian_block(g.n, 5, 42)
    W = w.apply(torch.as_tensor(V, device="cuda")).cpu().numpy()
    assert relerr(W, walks.apply_laplacian(phi, V)) <= TOL
    U0 = wlgen.unit_block(g.n, np.array([3, 100]))
    U = w.expmv(torch.as_tensor(U0, device="cuda"), [0.5, 3.0]).cpu().numpy()
    want = walks.diffusion(walks.walk_laplacian(phi), U0, [0.5, 3.0])
    for t in range(2):
        assert relerr(U[t], want[t]) <= TOL
    P = w.markov(torch.as_tensor(U0, device="cuda"), [4]).cpu().numpy()[0]
    assert relerr(P, walks.markov_evolve(phi, U0, [4])[0]) <= TOL
    w.close()


def test_exp_on_a_tree_with_nbt_walks():
    """On a tree the nonbacktracking counts vanish beyond the diameter, so the
    NBT series is a polynomial in A; the library's result still matches the
    oracle's series."""
    g = wlgen.path(25)
    A = dense(g)
    w = WL(g, variant="nbt", beta=0.9)
    phi = walks.phi_series(A, 1.0, walks.exp_coeffs(0.9))
    assert relerr(w.degrees().cpu().numpy(), walks.walk_degrees(phi)) <= TOL
    w.close()


@pytest.mark.parametrize("mu", [0.0, 1.0])
def test_exp_walk_degrees_of_a_large_star_closed_form(mu):
    """Star with m = 40000 leaves, beta = 1 / lambda_max(A) = 1 / sqrt(m), beyond
    the dense oracle's sizes. mu = 0: exp(beta A) acts on span{e_hub, leaves / sqrt(m)}
    as cosh(c) I + sinh(c) J with c = beta sqrt(m) = 1, so D_f(hub) = cosh c +
    sqrt(m) sinh c and D_f(leaf) = cosh c + sinh c / sqrt(m). The raw walk counts
    A^k 1 reach 200^k at the hub and leave the FP32 exponent range after 17
    terms; the series must carry the bounded terms c_k A^k 1 instead. mu = 1: a
    tree has no nonbacktracking walks of length 3 or more, so phi = I + beta A +
    (beta^2 / 2)(A^2 - D): D_f(hub) = 1 + beta m, D_f(leaf) = 1 + beta + (beta^2 / 2)(m - 1)."""
    from paper_2601_11338_gb300.api import WalkLaplacian
    m = 40000
    g = wlgen.star(m)
    variant = "allwalk" if mu == 0.0 else "nbt"
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant=variant, f="exp", prec="refined")
    beta = w.info["beta"]
    assert abs(beta * np.sqrt(m) - 1.0) <= 1e-9
    Df = w.degrees().cpu().numpy()
    w.close()
    deg = np.diff(g.row_ptr)
    hub = int(np.argmax(deg))
    leaves = np.arange(g.n) != hub
    if mu == 0.0:
        c = beta * np.sqrt(m)
        want_hub, want_leaf = np.cosh(c) + np.sqrt(m) * np.sinh(c), np.cosh(c) + np.sinh(c) / np.sqrt(m)
    else:
        want_hub, want_leaf = 1.0 + beta * m, 1.0 + beta + 0.5 * beta * beta * (m - 1)
    assert abs(Df[hub] - want_hub) <= 1e-12 * want_hub, (Df[hub], want_hub)
    assert np.abs(Df[leaves] - want_leaf).max() <= 1e-12 * want_leaf


def test_exp_edge_cases():
    """No edges: phi = I (only c_0 q_0 survives), D_f = 1, L = 0. An overflowing
    scale is reported as non-finite, not returned as garbage."""
    from paper_2601_11338_gb300 import wl
    from paper_2601_11338_gb300.api import WalkLaplacian
    n = 7
    w = WalkLaplacian(np.zeros(n + 1, np.int32), np.zeros(0, np.int32), n, f="exp", beta=0.7)
    np.testing.assert_allclose(w.degrees().cpu().numpy(), np.ones(n), rtol=0, atol=1e-15)
    V = torch.randn(n, 3, dtype=torch.float64, device="cuda")
    # phi V is V carried through the double-float series (48-bit significand)
    assert float(w.apply(V).abs().max()) <= 1e-14 * float(V.abs().max())
    w.close()
    g = wlgen.erdos_renyi(200, 12, 9)
    w = WL(g, beta=200.0)
    with pytest.raises(wl.WLError) as e:
        w.degrees()
    assert e.value.status == wl.WL_ERR_NONFINITE
    w.close()
