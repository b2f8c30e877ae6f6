"""Discrete-time diffusion (Sec. 3.3, Eq. let_there_be_markov with D = the
walk degrees): the CUDA chain through the C ABI against the CPU FP64 oracle.

Tolerances as for the other single-graph paths: relative 2-norm and largest element-wise error (relative to the column's largest entry) per column,
1e-10 for the FP64 form and 1e-8 for the refined form.
"""
import numpy as np
import pytest

import wlgen
from oracle import graph, walks
from parity_metrics import relerr  # max of norm-wise and element-wise error per column

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "refined": 1e-8}
STEPS = [0, 1, 2, 7, 20]


def dense(g):
    return graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)


def WL(g, **kw):
    from paper_2601_11338_gb300.api import WalkLaplacian
    return WalkLaplacian(g.row_ptr[:].astype(np.int32), g.col_idx, g.n, **kw)


def point_masses(n, nodes):
    P0 = np.zeros((n, len(nodes)))
    P0[nodes, np.arange(len(nodes))] = 1.0
    return P0


@pytest.mark.parametrize("prec", ["fp64", "refined"])
@pytest.mark.parametrize("variant,mu", [("allwalk", 0.0), ("nbt", 1.0), ("btdw", 0.5)])
@pytest.mark.parametrize("reorder", [0, 1])
def test_chain_matches_oracle(prec, variant, mu, reorder):
    g = wlgen.erdos_renyi(400, 7, 31)
    A = dense(g)
    w = WL(g, variant=variant, mu=mu, alpha_rel=0.5, prec=prec, tol=1e-13 if prec == "fp64" else 1e-11,
           reorder=reorder)
    phi = walks.phi_resolvent_closed(A, mu, w.info["alpha"])
    P0 = point_masses(g.n, [0, 17, 399])
    P0[:, 2] = wlgen.gaussian_block(g.n, 1, 4)[:, 0] ** 2  # a spread-out start
    P0[:, 2] /= P0[:, 2].sum()
    got = w.markov(torch.as_tensor(P0, device="cuda"), STEPS).cpu().numpy()
    want = walks.markov_evolve(phi, P0, STEPS)
    for t in range(len(STEPS)):
        assert relerr(got[t], want[t]) <= TOL[prec], (t, STEPS[t])
    w.close()


def test_identity_function_is_the_simple_random_walk():
    """phi = A, D_f = d: P = D^{-1} A. On the cycle C_n a walk from node 0
    is at offset j after s < n/2 steps with probability C(s, (s+j)/2) / 2^s."""
    from math import comb
    n = 64
    g = wlgen.cycle(n)
    w = WL(g, f="identity")
    got = w.markov(torch.as_tensor(point_masses(n, [0]), device="cuda"), [9]).cpu().numpy()[0][:, 0]
    want = np.zeros(n)
    for j in range(-9, 10):
        if (9 + j) % 2 == 0:
            want[j % n] = comb(9, (9 + j) // 2) / 2 ** 9
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    w.close()


def test_mass_nonnegativity_and_stationary_limit_at_size():
    """Chung-Lu n = 2e5, NBT, refined: 1^T p = 1 up to the solves' tolerance
    (exact solves conserve it; each step's residual, relative tol, can move
    the mass by at most sqrt(n) tol), p >= 0 up to the same, and a long run
    approaches pi = D_f / 1^T D_f (the chain's stationary distribution) on the
    nodes reachable from the start."""
    tol = 1e-11
    g = wlgen.chung_lu(200_000, seed=20260501)
    w = WL(g, variant="nbt", alpha_rel=0.5, prec="refined", tol=tol)
    nodes = wlgen.point_sources(g, 4, 20260502)
    P0 = torch.as_tensor(point_masses(g.n, nodes), device="cuda")
    steps = [1, 5, 50]
    P = w.markov(P0, steps).cpu().numpy()
    for t, s in enumerate(steps):
        np.testing.assert_allclose(P[t].sum(axis=0), 1.0, rtol=0, atol=s * np.sqrt(g.n) * tol)
        assert P[t].min() >= -s * tol
    Df = w.degrees().cpu().numpy()
    # the mass stays on the start's component; compare there
    for c in range(4):
        p = P[2][:, c]
        comp = p > 1e-300
        pi = Df[comp] / Df[comp].sum()
        assert np.abs(p[comp] - pi).sum() < np.abs(P[0][:, c][comp] - pi).sum()
    w.close()


def test_argument_checks():
    from paper_2601_11338_gb300 import wl
    g = wlgen.erdos_renyi(50, 4, 3)
    w = WL(g)
    P0 = torch.zeros((g.n, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((2, g.n, 2), dtype=torch.float64, device="cuda")
    for steps in ([3, 1], [-1, 2]):
        with pytest.raises(wl.WLError):
            wl.wl_markov(w.h, P0, 2, 2, steps, out, 2)
    w.close()


def test_edge_cases():
    """Zero steps return the start; k = 0 is a no-op; a graph without edges
    keeps every distribution where it is (phi = I, D_f = 1)."""
    g = wlgen.erdos_renyi(120, 5, 8)
    w = WL(g, variant="nbt", alpha_rel=0.5)
    P0 = point_masses(g.n, [5, 9])
    got = w.markov(torch.as_tensor(P0, device="cuda"), [0, 0]).cpu().numpy()
    np.testing.assert_array_equal(got[0], P0)
    np.testing.assert_array_equal(got[1], P0)
    out = torch.empty((1, g.n, 0), dtype=torch.float64, device="cuda")
    from paper_2601_11338_gb300 import wl
    assert wl.wl_markov(w.h, torch.empty((g.n, 0), dtype=torch.float64, device="cuda"), 0, 0, [3], out, 0) == wl.WL_OK
    w.close()
    n = 9
    from paper_2601_11338_gb300.api import WalkLaplacian
    w0 = WalkLaplacian(np.zeros(n + 1, np.int32), np.zeros(0, np.int32), n, alpha=0.3)
    P0 = point_masses(n, [1, 4])
    got = w0.markov(torch.as_tensor(P0, device="cuda"), [3]).cpu().numpy()[0]
    np.testing.assert_allclose(got, P0, rtol=0, atol=1e-15)
    w0.close()
