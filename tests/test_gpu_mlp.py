"""Learned warm start: features, network gradients, Adam step and inference
on the GPU against the FP64 oracle; then the warm start's effect on the
walk-degree solve.

Tolerances: features are FP32 roundings of FP64 values (relative 1e-6,
triangle counts exact); the gradient accumulates in FP32 over 128 rows and
in FP64 across them (relative 1e-5 against the FP64 analytic gradient,
1e-4 against central differences); one Adam step relative 1e-5.
"""
import numpy as np
import pytest

import wlgen
from oracle import features, graph, mlp, walks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def flatten(p):
    """oracle parameter dict -> the library's parameter vector (mean 0, std 1)."""
    return np.concatenate([np.zeros(4), np.ones(4), p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"],
                           p["W3"].ravel(), p["b3"]]).astype(np.float32)


def unflatten(v, H=64):
    v = v.astype(np.float64)
    o = 8
    out = {}
    for name, shape in (("W1", (H, 4)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (1, H)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = v[o:o + size].reshape(shape)
        o += size
    return out


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("reorder", [0, 1])
def test_features_match_oracle(reorder):
    from paper_2601_11338_gb300.api import WalkLaplacian, mlp_features
    for g, variant, mu in ((wlgen.erdos_renyi(600, 12.0, 31), "nbt", 1.0),
                           (wlgen.barabasi_albert(500, 4, 32), "btdw", 0.5),
                           (wlgen.grid2d(12, 17), "allwalk", 0.0),
                           (wlgen.complete(30), "nbt", 1.0)):
        w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant=variant, mu=mu, alpha_rel=0.5,
                          reorder=reorder)
        F, X = mlp_features(w)
        F = F.cpu().numpy().astype(np.float64)
        X = X.cpu().numpy()
        A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
        ref = features.raw_features(A)
        assert rel(F, ref) <= 1e-6
        tri = features.triangles_by_intersection(g.row_ptr, g.col_idx, g.n)
        assert np.array_equal(np.rint(np.expm1(F[:, 2])), tri)
        # x_an = 1 + B 1 + B^2 1, B = (alpha A - alpha^2 mu D) / (1 - mu^2 alpha^2)
        alpha = w.info["alpha"]
        a = 1.0 - mu * mu * alpha * alpha
        B = (alpha * A - alpha * alpha * mu * np.diag(A.sum(1))) / a
        one = np.ones(g.n)
        assert rel(X, one + B @ one + B @ (B @ one)) <= 1e-13
        w.close()


def test_gradient_matches_oracle_and_central_differences():
    from paper_2601_11338_gb300 import wl
    rng = np.random.default_rng(41)
    p = mlp.init_params(64, 4, seed=3)
    X = rng.normal(size=(300, 4))
    t = rng.normal(size=300)
    v = flatten(p)
    Xf = X.astype(np.float32)
    tf = t.astype(np.float32)
    grad = np.zeros(v.size, dtype=np.float32)
    loss = wl.wl_mlp_loss_grad(v, Xf, tf, 300, grad)
    # the oracle on the same FP32-rounded inputs and weights
    p32 = unflatten(v)
    X32, t32 = Xf.astype(np.float64), tf.astype(np.float64)
    g_ref = mlp.backward(p32, X32, t32)
    assert abs(loss - mlp.loss(p32, X32, t32)) <= 1e-6 * mlp.loss(p32, X32, t32)
    g_gpu = unflatten(grad)
    for k in mlp.NAMES:
        assert rel(g_gpu[k], g_ref[k]) <= 1e-5, k
    # central differences on a smaller network slice: the first-layer weights
    g_num = mlp.numerical_grad(p32, X32, t32, h=1e-5)
    for k in ("W1", "b1", "W3", "b3"):
        assert rel(g_gpu[k], g_num[k]) <= 1e-4, k


def test_adam_step_matches_oracle():
    from paper_2601_11338_gb300 import wl
    rng = np.random.default_rng(42)
    p = mlp.init_params(64, 4, seed=4)
    X = rng.normal(size=(513, 4)).astype(np.float32)
    t = rng.normal(size=513).astype(np.float32)
    v = flatten(p)
    v0 = v.copy()
    wl.wl_mlp_train(v, X, t, 513, 1, 0, 1e-3, 0)
    p32 = unflatten(v0)
    g = mlp.backward(p32, X.astype(np.float64), t.astype(np.float64))
    want = mlp.adam_step(p32, g, {}, lr=1e-3)
    got = unflatten(v)
    for k in mlp.NAMES:
        assert rel(got[k] - unflatten(v0)[k], want[k] - unflatten(v0)[k]) <= 1e-4, k


def test_predict_matches_oracle_forward_with_standardisation():
    from paper_2601_11338_gb300 import wl
    rng = np.random.default_rng(43)
    p = mlp.init_params(64, 4, seed=5)
    v = flatten(p)
    v[0:4] = [0.5, -1.0, 2.0, 0.25]
    v[4:8] = [2.0, 0.5, 1.5, 3.0]
    F = rng.normal(size=(1000, 4)).astype(np.float32)
    xan = rng.uniform(1.0, 3.0, size=1000)
    out = np.empty(1000)
    wl.wl_mlp_predict(v, F, 1000, xan, out)
    Z = (F.astype(np.float64) - v[0:4].astype(np.float64)) / v[4:8].astype(np.float64)
    y, _ = mlp.forward(unflatten(v), Z)
    assert rel(out, xan * np.exp(y)) <= 1e-5


def test_training_reduces_loss_and_warm_start_cuts_iterations():
    """Trained on walk degrees of small ER / Chung-Lu / BA / grid graphs, the
    network's guess x0 = x_an exp(y) on a held-out Chung-Lu graph is closer
    to D_f than the analytic two-term guess x_an, and the NBT walk-degree CG
    started from it needs fewer iterations than from x = 0. (The analytic
    guess, whose error is a smooth Krylov remainder, still needs fewer
    iterations than the learned one; the test records all three.)"""
    from paper_2601_11338_gb300 import warmstart, wl
    from paper_2601_11338_gb300.api import WalkLaplacian, mlp_features
    train = [wlgen.erdos_renyi(3000, 10.0, 51), wlgen.chung_lu(5000, seed=52), wlgen.barabasi_albert(4000, 3, 53),
             wlgen.grid2d(50, 60), wlgen.chung_lu(8000, seed=54), wlgen.erdos_renyi(6000, 6.0, 55)]
    F, T = warmstart.training_rows(train, "nbt")
    p0 = warmstart.initial_params(0)
    p = p0.copy()
    loss0 = wl.wl_mlp_loss_grad(p0, F, T, F.shape[0], np.zeros(p0.size, dtype=np.float32))
    loss = wl.wl_mlp_train(p, F, T, F.shape[0], 1500, 0, 3e-3, 1)
    assert loss < 0.5 * loss0
    g = wlgen.chung_lu(20000, seed=56)
    iters, err = {}, {}
    Dref = None
    for mode in ("cold", "analytic", "mlp"):
        w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5, prec="fp64",
                          tol=1e-10)
        Fg, X = mlp_features(w)
        x0 = None
        if mode == "analytic":
            wl.wl_set_warm_start(w.h, X)
            x0 = X
        elif mode == "mlp":
            wl.wl_mlp_warm_start(w.h, p)
            x0 = torch.empty_like(X)
            wl.wl_mlp_predict(p, Fg, g.n, X, x0)
        D = w.degrees()
        iters[mode] = w.last.iters
        if mode == "cold":
            Dref = D.clone()
        else:
            assert rel(D.cpu().numpy(), Dref.cpu().numpy()) <= 1e-9
            err[mode] = rel(x0.cpu().numpy(), Dref.cpu().numpy())
        w.close()
    print("walk-degree CG iterations", iters, "guess errors", err)
    assert err["mlp"] < err["analytic"]
    assert iters["mlp"] < iters["cold"]
