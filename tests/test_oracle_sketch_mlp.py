"""Pins for the oracle's trace estimator, Philox generator, warm-start MLP
and node features (no GPU)."""
import numpy as np
import pytest

import wlgen
from oracle import features, graph, mlp, philox, spectral, walks, xnys


# ---------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    """Published known-answer vectors of Philox4x32-10 (Salmon et al., SC'11,
    reference distribution): counter/key all zero, all ones, and pi digits."""
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for c, k, want in cases:
        got = philox.philox4x32_10(np.array([c], np.uint32), np.array([k], np.uint32))[0]
        assert [int(x) for x in got] == want


def test_bf16_rounding_is_nearest_even():
    # bf16 keeps 7 fraction bits: the spacing at 1.0 is 2^-7, a tie sits at 2^-8
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, 1.0 + 2 ** -9,
                  -2.5, 1.0 + 2 ** -8 + 2 ** -40])
    b = philox.to_bf16_bits(x)
    v = philox.bf16_bits_to_f64(b)
    assert v[0] == 1.0
    assert v[1] == 1.0                            # tie -> even (down)
    assert v[2] == 1.0 + 2 ** -6                  # tie -> even (up)
    assert v[3] == 1.0 + 2 ** -7                  # above the tie -> up
    assert v[4] == 1.0                            # below the tie -> down
    assert v[6] == 1.0 + 2 ** -7                  # FP64 above a tie that FP32 would create
    assert v[5] == -2.5
    rng = np.random.default_rng(0)
    y = rng.standard_normal(10000) * 10 ** rng.uniform(-5, 5, 10000)
    vy = philox.bf16_bits_to_f64(philox.to_bf16_bits(y))
    ulp = 2.0 ** (np.floor(np.log2(np.abs(y))) - 7)
    assert (np.abs(vy - y) <= 0.5 * ulp + 1e-300).all()


def test_gaussian_sketch_moments():
    v, _ = philox.gaussian_sketch(4096, 64, 123)
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1) < 0.01
    c = np.corrcoef(v[:, :8].T)
    assert np.abs(c - np.eye(8)).max() < 0.06


# ---------------------------------------------------------------- XNysTrace
def test_xnystrace_exact_for_low_rank_psd():
    """The Nystrom approximation from M - 1 vectors reproduces a PSD matrix of
    rank <= M - 1 exactly, so every t_i equals the trace."""
    rng = np.random.default_rng(3)
    n, r, M = 60, 5, 8
    G = rng.standard_normal((n, r))
    A = G @ G.T
    Om = rng.standard_normal((n, M))
    est, err, t = xnys.xnystrace(A, Om)
    assert abs(est - np.trace(A)) < 1e-9 * np.trace(A)
    assert err < 1e-9 * np.trace(A)


def test_xnystrace_two_vector_closed_form():
    """M = 2: A_hat_(1) = y2 y2^T / (w2^T y2), so
    t_1 = |y2|^2 / (w2^T y2) + w1^T A w1 - (w1^T y2)^2 / (w2^T y2)."""
    rng = np.random.default_rng(4)
    G = rng.standard_normal((10, 10))
    A = G @ G.T + np.eye(10)
    Om = rng.standard_normal((10, 2))
    est, err, t = xnys.xnystrace(A, Om)
    w1, w2 = Om[:, 0], Om[:, 1]
    y1, y2 = A @ w1, A @ w2
    t1 = y2 @ y2 / (w2 @ y2) + w1 @ y1 - (w1 @ y2) ** 2 / (w2 @ y2)
    t2 = y1 @ y1 / (w1 @ y1) + w2 @ y2 - (w2 @ y1) ** 2 / (w1 @ y1)
    np.testing.assert_allclose(t, [t1, t2], rtol=1e-12)
    np.testing.assert_allclose(err, abs(t1 - t2) / 2, rtol=1e-12)


def test_xnystrace_unbiased_on_walk_resolvent():
    """Each t_i is unbiased for tr(A) with Gaussian test vectors; the mean of
    many independent estimates lands within a few standard errors."""
    g = wlgen.erdos_renyi(60, 6, 5)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    alpha = 0.5 / spectral.lambda_max(A)
    phi = walks.phi_allwalk_resolvent_eig(A, alpha)
    tr = xnys.exact_trace(phi)
    rng = np.random.default_rng(5)
    ests = [xnys.xnystrace(phi, rng.standard_normal((60, 6)))[0] for _ in range(150)]
    se = np.std(ests, ddof=1) / np.sqrt(len(ests))
    assert abs(np.mean(ests) - tr) < 4 * se + 1e-12


# ---------------------------------------------------------------- MLP
def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    p = mlp.init_params(H=8, seed=1)
    X = rng.standard_normal((16, 4))
    t = rng.standard_normal(16)
    ga = mlp.backward(p, X, t)
    gn = mlp.numerical_grad(p, X, t)
    for k in mlp.NAMES:
        np.testing.assert_allclose(ga[k], gn[k], rtol=1e-6, atol=1e-9)


def test_adam_first_step_is_signed_learning_rate():
    """At t = 1 the bias corrections give m_hat = g and v_hat = g^2, so the
    update is lr * g / (|g| + eps)."""
    p = {k: np.ones(3) for k in mlp.NAMES}
    g = {k: np.array([0.5, -2.0, 1e-3]) for k in mlp.NAMES}
    q = mlp.adam_step({k: v.copy() for k, v in p.items()}, g, {}, lr=0.1)
    for k in mlp.NAMES:
        np.testing.assert_allclose(q[k], 1 - 0.1 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12)


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((256, 4))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    p = mlp.init_params(H=16, seed=2)
    st = {}
    l0 = mlp.loss(p, X, t)
    for _ in range(300):
        p = mlp.adam_step(p, mlp.backward(p, X, t), st, lr=1e-2)
    assert mlp.loss(p, X, t) < 0.2 * l0


# ---------------------------------------------------------------- features
def test_features_closed_forms():
    """K_5: d = 4, A d = 16, 6 triangles per node, 4 * 3 = 12 NBT 2-walks.
    C_n (n > 3): no triangles, 2 NBT 2-walks."""
    A = graph.dense_adjacency(*(lambda g: (g.row_ptr, g.col_idx, g.n))(wlgen.complete(5)))
    f = features.raw_features(A)
    np.testing.assert_allclose(f[0], np.log1p([4, 16, 6, 12]))
    g = wlgen.cycle(9)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    f = features.raw_features(A)
    np.testing.assert_allclose(f[0], np.log1p([2, 4, 0, 2]))


def test_triangles_two_ways():
    g = wlgen.erdos_renyi(80, 10, 8)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    np.testing.assert_allclose(np.expm1(features.raw_features(A)[:, 2]),
                               features.triangles_by_intersection(g.row_ptr, g.col_idx, g.n), atol=1e-9)


# ---------------------------------------------------------------- average return probability
def test_return_probability_cycle_closed_form():
    """On C_n with the combinatorial Laplacian the eigenvalues are
    2 - 2 cos(2 pi j / n), and by Poisson summation
    tr(exp(-t L)) / n = e^{-2t} sum_m I_{m n}(2t) (modified Bessel functions);
    for n = 40 and t <= 3 the terms |m| >= 2 are below 1e-30."""
    from scipy.special import iv
    n = 40
    A = graph.dense_adjacency(*_cycle_csr(n), n)
    L = np.diag(A.sum(axis=1)) - A
    ts = [0.0, 0.1, 1.0, 3.0]
    got = xnys.return_probability(L, ts)
    want = [np.exp(-2 * t) * (iv(0, 2 * t) + 2 * iv(n, 2 * t)) for t in ts]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def test_return_probability_limits():
    """p(0) = 1; for large t only the null space of L survives: p -> c / n
    with c connected components (two here)."""
    A = np.zeros((7, 7))
    for i, j in [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 6)]:
        A[i, j] = A[j, i] = 1.0
    L = np.diag(A.sum(axis=1)) - A
    p = xnys.return_probability(L, [0.0, 200.0])
    assert abs(p[0] - 1.0) < 1e-15
    assert abs(p[1] - 2.0 / 7.0) < 1e-12


@pytest.mark.parametrize("which", ["grid", "er"])
def test_return_probability_grows_with_mu_for_exp(which):
    """Sec. 4.4 (figure on varying mu): for the BTDW exponential Laplacian
    L_mu(exp) the average return probability rises as mu grows from 0 (all
    walks) to 1 (nonbacktracking), since suppressing backtracks slows the
    spreading. Checked on a grid (a road-network-like stand-in) and an ER
    graph at beta = 1 / lambda_max(A), t in (0, 5]; the mu = 0 end equals the
    all-walk exponential by eigendecomposition."""
    if which == "grid":
        g = wlgen.grid2d(8, 10)
    else:
        g = wlgen.erdos_renyi(60, 5, 1)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    beta = 1.0 / spectral.lambda_max(A)
    ts = np.linspace(0.0, 5.0, 11)[1:]
    ps = []
    for mu in (0.0, 0.25, 0.5, 0.75, 1.0):
        phi = walks.phi_series(A, mu, walks.exp_coeffs(beta))
        ps.append(xnys.return_probability(walks.walk_laplacian(phi), ts))
    ps = np.array(ps)
    assert np.all(np.diff(ps, axis=0) > 0), np.diff(ps, axis=0).min()
    p0 = xnys.return_probability(walks.walk_laplacian(walks.phi_allwalk_exp_eig(A, beta)), ts)
    np.testing.assert_allclose(ps[0], p0, rtol=1e-12)


def _cycle_csr(n):
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    col = np.empty(2 * n, dtype=np.int32)
    for i in range(n):
        a, b = (i - 1) % n, (i + 1) % n
        col[2 * i], col[2 * i + 1] = min(a, b), max(a, b)
    return rp, col
