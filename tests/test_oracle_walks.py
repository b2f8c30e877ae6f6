"""Pins for the CPU FP64 oracle's walk functions, against what the paper and
the mathematics fix (no GPU)."""
import math
import os

import numpy as np
import pytest

import wlgen
from oracle import brute, graph, spectral, walks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "g58_fig1.txt")


def dense(g):
    return graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)


def small_graphs():
    rng = np.random.default_rng(11)
    B = np.triu((rng.random((7, 7)) < 0.45).astype(float), 1)
    B = B + B.T
    return {
        "rand7": B,
        "g58": dense(wlgen.g58()),
        "K4": dense(wlgen.complete(4)),
        "C5": dense(wlgen.cycle(5)),
    }


def load_fig1():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            panel, node, v = line.split()
            vals.setdefault(panel, {})[int(node)] = float(v)
    return vals


# ---------------------------------------------------------------- Fig. 1 pins
def _normalised(d):
    return d / d.sum()


@pytest.mark.parametrize("panel", ["L", "res", "exp", "nbtexp"])
def test_fig1_stationary_distributions(panel):
    """Fig. 1 (Sec. 5.1): stationary distributions of the chains induced by
    each Laplacian on G_{5,8}, printed to ~15 digits."""
    A = dense(wlgen.g58())
    want = load_fig1()[panel]
    if panel == "L":
        pi = _normalised(graph.degree_vector(A))
    elif panel == "res":
        alpha = 1.0 / (2.0 * spectral.lambda_max(A))
        phi = walks.phi_series(A, 0.0, walks.resolvent_coeffs(alpha))
        pi = walks.markov_stationary(phi)
        np.testing.assert_allclose(phi, walks.phi_allwalk_resolvent_eig(A, alpha), rtol=0, atol=1e-13)
    elif panel == "exp":
        phi = walks.phi_series(A, 0.0, walks.exp_coeffs(1.0))
        pi = walks.markov_stationary(phi)
    else:
        # L_1(exp): the printed values are reproduced by phi = sum_{j>=2} p_j / (j-1)!,
        # i.e. [O I] phi_1(Z) [A; A^2 - D] with c_0 = c_1 = 0 (reading of Eq.
        # exp-based-laplacian against its own figure).
        p = walks.nbt_counts(A, 30)
        phi = sum(p[j] / math.factorial(j - 1) for j in range(2, 31))
        pi = walks.markov_stationary(phi)
        # on this tree the entries are rationals with denominator 674
        np.testing.assert_allclose(pi * 674, np.round(pi * 674), atol=1e-10)
    for node, v in want.items():
        assert abs(pi[node - 1] - v) <= 2e-14 + 1e-12 * v, (panel, node, pi[node - 1], v)
    for leaf in range(6, 14):  # leaves share the value of node 6
        assert abs(pi[leaf - 1] - want[6]) <= 1e-13


# ---------------------------------------------------------------- walk counts
@pytest.mark.parametrize("name", ["rand7", "g58", "K4", "C5"])
@pytest.mark.parametrize("mu", [0.0, 0.25, 0.5, 1.0])
def test_btdw_counts_match_brute_force(name, mu):
    """Eq. qrec against explicit enumeration of walks weighted by
    (1 - mu)^{#backtracking steps} (Sec. 3.2)."""
    A = small_graphs()[name]
    kmax = 5 if name != "g58" else 4
    q = walks.btdw_counts(A, mu, kmax)
    for k in range(kmax + 1):
        np.testing.assert_allclose(q[k], brute.weighted_walk_counts(A, k, mu), rtol=0, atol=1e-9)


def test_nbt_counts_are_btdw_at_mu_one_and_powers_at_zero():
    """Eq. qrec reduces to Prop. power-of-adjacency at mu = 0 and to Eq. Br at mu = 1."""
    A = small_graphs()["rand7"]
    p = walks.nbt_counts(A, 7)
    q1 = walks.btdw_counts(A, 1.0, 7)
    q0 = walks.btdw_counts(A, 0.0, 7)
    for k in range(8):
        np.testing.assert_array_equal(p[k], q1[k])
        np.testing.assert_array_equal(q0[k], np.linalg.matrix_power(A, k))


# ---------------------------------------------------------------- phi two ways
@pytest.mark.parametrize("mu", [0.0, 0.3, 0.75, 1.0])
@pytest.mark.parametrize("frac", [0.2, 0.5, 0.9])
def test_resolvent_closed_form_equals_series(mu, frac):
    """sum_k alpha^k q_k = (1 - mu^2 alpha^2) M_mu(alpha)^{-1}
    (Eq. deformed at mu = 1 and its general-mu extension), for alpha inside
    the radius 1 / rho(Z) of Prop. whe-we-converge."""
    A = small_graphs()["rand7"]
    rho = spectral.rho_companion(A, mu)
    alpha = frac / rho
    series = walks.phi_series(A, mu, walks.resolvent_coeffs(alpha))
    closed = walks.phi_resolvent_closed(A, mu, alpha)
    np.testing.assert_allclose(series, closed, rtol=0, atol=1e-12 * np.abs(closed).max())
    if mu == 0.0:
        np.testing.assert_allclose(closed, walks.phi_allwalk_resolvent_eig(A, alpha), atol=1e-13)


def test_deformed_laplacian_identity_mu_one():
    """Eq. deformed: phi [I - alpha A - alpha^2 (I - D)] = (1 - alpha^2) I."""
    A = small_graphs()["rand7"]
    alpha = 0.4 / spectral.rho_companion(A, 1.0)
    n = A.shape[0]
    D = np.diag(A.sum(1))
    phi = walks.phi_series(A, 1.0, walks.resolvent_coeffs(alpha))
    lhs = phi @ (np.eye(n) - alpha * A - alpha ** 2 * (np.eye(n) - D))
    np.testing.assert_allclose(lhs, (1 - alpha ** 2) * np.eye(n), atol=1e-13)


def test_exp_series_equals_spectral_form():
    A = small_graphs()["rand7"]
    beta = 1.0 / spectral.lambda_max(A)
    np.testing.assert_allclose(walks.phi_series(A, 0.0, walks.exp_coeffs(beta)),
                               walks.phi_allwalk_exp_eig(A, beta), atol=1e-13)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("mu", [0.0, 0.5, 1.0])
def test_laplacian_invariants(mu):
    """Props. still-an-mmatrix / still-again-an-mmatrix and Lemma
    being_an_m_matrix: symmetric, L 1 = 0, nonpositive off-diagonal, PSD."""
    A = dense(wlgen.erdos_renyi(40, 5, 3))
    alpha = 0.5 / spectral.rho_companion(A, mu)
    phi = walks.phi_resolvent_closed(A, mu, alpha)
    assert (phi >= -1e-15).all()
    L = walks.walk_laplacian(phi)
    Df = walks.walk_degrees(phi)
    assert np.abs(L @ np.ones(40)).max() <= 1e-14 * Df.max()
    np.testing.assert_allclose(L, L.T, atol=1e-15)
    off = L - np.diag(np.diag(L))
    assert off.max() <= 1e-15
    assert np.linalg.eigvalsh(L)[0] >= -1e-12


def test_diffusion_conserves_mass_and_stays_nonnegative():
    """Sec. 2.1 and 3.2: with an M-matrix Laplacian the evolution conserves
    1^T u and keeps u >= 0; it equilibrates to a multiple of 1."""
    A = dense(wlgen.erdos_renyi(50, 6, 4))
    alpha = 0.5 / spectral.rho_companion(A, 1.0)
    L = walks.walk_laplacian(walks.phi_resolvent_closed(A, 1.0, alpha))
    U0 = np.zeros((50, 2)); U0[3, 0] = 1.0; U0[7, 1] = 2.0
    taus = [0.1, 1.0, 10.0, 1e4]
    U = walks.diffusion(L, U0, taus)
    lam = np.linalg.eigvalsh(L)
    for t, Ut in zip(taus, U):
        # rounding of the zero eigenvalue grows like tau * eps * |L|
        np.testing.assert_allclose(Ut.sum(0), U0.sum(0), rtol=1e-14 * max(1.0, t * lam[-1]))
        assert Ut.min() >= -1e-14
    # connected? then the limit is the mean
    if lam[1] > 1e-8:
        np.testing.assert_allclose(U[-1], np.ones((50, 1)) * U0.mean(0), atol=1e-10)


# ---------------------------------------------------------------- reductions
def test_identity_function_gives_combinatorial_laplacian():
    """c = (0, 1, 0, ...) gives L(c) = D - A (Sec. 3.1)."""
    A = small_graphs()["rand7"]
    phi = walks.phi_series(A, 0.0, lambda k: 1.0 if k == 1 else 0.0)
    np.testing.assert_array_equal(walks.walk_laplacian(phi), graph.combinatorial_laplacian(A))


def test_mu_zero_is_all_walk():
    """L_0(c) = L(c) (Sec. 3.2.1)."""
    A = small_graphs()["rand7"]
    alpha = 0.5 / spectral.lambda_max(A)
    np.testing.assert_allclose(walks.phi_resolvent_closed(A, 0.0, alpha),
                               walks.phi_allwalk_resolvent_eig(A, alpha), atol=1e-13)


@pytest.mark.parametrize("mu", [0.0, 1.0])
def test_small_alpha_limit_is_combinatorial_laplacian(mu):
    """L(alpha) / alpha -> D - A as alpha -> 0 (q_1 = A), error O(alpha)."""
    A = small_graphs()["rand7"]
    L0 = graph.combinatorial_laplacian(A)
    errs = []
    for alpha in (1e-3, 1e-4, 1e-5):
        L = walks.walk_laplacian(walks.phi_resolvent_closed(A, mu, alpha))
        errs.append(np.abs(L / alpha - L0).max())
    assert 7 < errs[0] / errs[1] < 13 and 7 < errs[1] / errs[2] < 13


# ---------------------------------------------------------------- closed forms on regular graphs
@pytest.mark.parametrize("mu", [0.0, 0.5, 1.0])
def test_torus_closed_forms(mu):
    """On a d-regular graph M_mu(alpha) = (a + alpha^2 mu d) I - alpha A shares A's
    eigenvectors: D_f = a / (a + alpha^2 mu d - alpha d) 1, and L has the
    eigenvalues f(d) - f(lambda), so exp(-tau L) e_1 is a cosine sum. The
    eigenvalues of Z solve z^2 - lambda z + mu (d - mu) = 0 (Eq. Zdef), so
    rho(Z_mu) = d - mu when d > 2 mu. Here the r x c torus, d = 4, with
    lambda_jk = 2 cos(2 pi j / r) + 2 cos(2 pi k / c)."""
    r, c, d = 5, 6, 4
    A = dense(wlgen.torus2d(r, c))
    rho = spectral.rho_companion(A, mu)
    assert abs(rho - (d - mu)) < 1e-9
    alpha = 0.5 / rho
    a = 1 - mu * mu * alpha * alpha
    phi = walks.phi_resolvent_closed(A, mu, alpha)
    np.testing.assert_allclose(walks.walk_degrees(phi), a / (a + alpha ** 2 * mu * d - alpha * d), rtol=1e-14)
    f = lambda lam: a / (a + alpha ** 2 * mu * d - alpha * lam)
    j = np.arange(r)[:, None]
    k = np.arange(c)[None, :]
    lam = 2 * np.cos(2 * np.pi * j / r) + 2 * np.cos(2 * np.pi * k / c)
    ev = f(d) - f(lam)
    tau = 3.0
    want = np.array([[np.mean(np.exp(-tau * ev) * np.cos(2 * np.pi * j * m1 / r) * np.cos(2 * np.pi * k * m2 / c))
                      for m2 in range(c)] for m1 in range(r)]).ravel()
    U0 = np.zeros((r * c, 1)); U0[0, 0] = 1
    got = walks.diffusion(walks.walk_laplacian(phi), U0, [tau])[0][:, 0]
    np.testing.assert_allclose(got, want, atol=1e-15)


# ---------------------------------------------------------------- spectral
@pytest.mark.parametrize("mu", [0.0, 0.4, 1.0])
def test_first_singular_t_is_inverse_rho(mu):
    """M_mu(t) is positive definite on [0, 1/rho(Z_mu)) and singular at its end
    (Prop. CGworks and the remark extending it to mu in [0, 1])."""
    A = dense(wlgen.erdos_renyi(30, 5, 9))
    rho = spectral.rho_companion(A, mu)
    t = spectral.first_singular_t(A, mu)
    assert abs(t * rho - 1) < 1e-9
    if mu == 0.0:
        assert abs(rho - spectral.lambda_max(A)) < 1e-10


# ---------------------------------------------------------------- CPU Krylov restatement (Sec. 4)
@pytest.mark.parametrize("mu", [0.0, 1.0])
def test_cpu_krylov_matches_dense_definitions(mu):
    """CG on M (Sec. 4.2) and Lanczos exp(-tau T_m) (Sec. 4.1) reproduce the
    dense definitions: D_f = phi 1, L V, exp(-tau L) u0."""
    from oracle import krylov
    g = wlgen.erdos_renyi(300, 6, 21)
    A = dense(g)
    alpha = 0.5 / spectral.rho_companion(A, mu)
    phi = walks.phi_resolvent_closed(A, mu, alpha)
    L = walks.walk_laplacian(phi)
    op = krylov.ResolventLaplacian(krylov.adjacency(g.row_ptr, g.col_idx, g.n), mu, alpha, tol=1e-14)
    np.testing.assert_allclose(op.Df, walks.walk_degrees(phi), rtol=1e-12)
    V = np.random.default_rng(0).standard_normal((g.n, 3))
    np.testing.assert_allclose(op.apply(V), L @ V, rtol=0, atol=1e-11 * np.abs(L @ V).max())
    u0 = np.zeros(g.n); u0[4] = 1.0
    U, m = krylov.lanczos_expmv(op.apply, u0, [0.1, 1.0, 10.0], tol=1e-12)
    want = walks.diffusion(L, u0[:, None], [0.1, 1.0, 10.0])
    for u, w in zip(U, want):
        assert np.linalg.norm(u - w[:, 0]) <= 1e-10 * np.linalg.norm(w)
    assert 0 < m <= 300


def test_cpu_lanczos_does_not_stop_on_a_vanished_approximation():
    """Near the pole (alpha = 0.998 / rho(Z_1)) the hub of a Chung-Lu graph has
    a walk degree in the hundreds, so for tau = 100 the first Ritz values all
    exceed 745 / tau and exp(-tau T_m) e_1 underflows to zero for the first
    few steps. Two zero approximations agree, but the exact result keeps the
    mass of u0 (L 1 = 0, Sec. 4.1): the run must go on until the slow modes
    enter the Krylov space, and then match the dense definition."""
    from oracle import krylov
    g = wlgen.chung_lu(1500, seed=7)
    A = dense(g)
    Asp = krylov.adjacency(g.row_ptr, g.col_idx, g.n)
    L = walks.walk_laplacian(walks.phi_resolvent_closed(A, 1.0, 0.998 / krylov.rho_companion_sparse(Asp, 1.0)))
    u0 = np.zeros(g.n)
    u0[int(np.argmax(A.sum(axis=1)))] = 1.0
    U, m = krylov.lanczos_expmv(lambda v: L @ v, u0, [100.0], tol=1e-10, m_max=1000)
    want = walks.diffusion(L, u0[:, None], [100.0])[0][:, 0]
    assert m > 100, m
    assert abs(U[0].sum() - 1.0) <= 1e-9
    assert np.linalg.norm(U[0] - want) <= 1e-9 * np.linalg.norm(want)


@pytest.mark.parametrize("mu", [0.0, 0.5, 1.0])
def test_sparse_companion_radius_matches_dense(mu):
    from oracle import krylov
    g = wlgen.erdos_renyi(200, 6, 22)
    A = dense(g)
    got = krylov.rho_companion_sparse(krylov.adjacency(g.row_ptr, g.col_idx, g.n), mu)
    assert abs(got - spectral.rho_companion(A, mu)) <= 1e-8 * got


# ---------------------------------------------------------------- discrete-time chain
def test_markov_evolve_simple_random_walk_on_cycle():
    """With phi = A (the combinatorial Laplacian D - A) the chain of Sec. 3.3 is
    the simple random walk: on C_n, from node 0, after s < n/2 steps the walk
    sits at offset j with probability C(s, (s + j)/2) / 2^s (j = s mod 2)."""
    n, s = 40, 13
    A = dense(wlgen.cycle(n))
    P0 = np.zeros((n, 1))
    P0[0, 0] = 1.0
    got = walks.markov_evolve(A, P0, [s])[0][:, 0]
    want = np.zeros(n)
    for j in range(-s, s + 1):
        if (s + j) % 2 == 0:
            want[j % n] = math.comb(s, (s + j) // 2) / 2 ** s
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-16)


@pytest.mark.parametrize("mu", [0.0, 0.5, 1.0])
def test_markov_evolve_conserves_mass_and_reaches_stationary(mu):
    """p_{s+1} = p_s P with P = D_f^{-1} phi: 1^T p is conserved (this fixes the
    orientation: P p would not conserve it on an irregular graph), p stays
    nonnegative, and the chain converges to the stationary distribution that
    Fig. 1 pins (markov_stationary)."""
    A = dense(wlgen.g58())
    alpha = 0.5 / spectral.rho_companion(A, mu) if mu > 0 else 0.5 / spectral.lambda_max(A)
    phi = walks.phi_resolvent_closed(A, mu, alpha)
    P0 = np.zeros((A.shape[0], 2))
    P0[0, 0] = 1.0
    P0[7, 1] = 1.0
    out = walks.markov_evolve(phi, P0, [1, 3, 400])
    for p in out:
        np.testing.assert_allclose(p.sum(axis=0), 1.0, rtol=0, atol=1e-14)
        assert p.min() >= 0.0
    pi = walks.markov_stationary(phi)
    for c in range(2):
        np.testing.assert_allclose(out[-1][:, c], pi, rtol=0, atol=1e-12)
    # the wrong orientation breaks conservation on this irregular graph
    P = phi / walks.walk_degrees(phi)[:, None]
    assert abs((P @ P0[:, 0]).sum() - 1.0) > 1e-3
