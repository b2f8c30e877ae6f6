"""FP64 reference for the warm-start network: a 3-layer perceptron
4 -> H -> H -> 1 with tanh hidden activations, mean squared error loss, and
the Adam update (Kingma and Ba, ICLR 2015). The paper has no learned part;
this network only predicts log walk degrees used as a CG starting guess.
Test infrastructure only.

Parameter layout (shared definition): W1 [H, 4], b1 [H], W2 [H, H], b2 [H],
W3 [1, H], b3 [1]; y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3.
Loss over a batch of B rows: L = (1/B) sum_b (y_b - t_b)^2.
"""
import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_params(H=64, n_in=4, seed=0):
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)

    def glorot(fo, fi):
        lim = np.sqrt(6.0 / (fi + fo))
        return rng.uniform(-lim, lim, size=(fo, fi))

    return {"W1": glorot(H, n_in), "b1": np.zeros(H), "W2": glorot(H, H), "b2": np.zeros(H),
            "W3": glorot(1, H), "b3": np.zeros(1)}


def forward(p, X):
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y[:, 0], (X, h1, h2)


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(np.mean((y - t) ** 2))


def backward(p, X, t):
    """Analytic gradient of the MSE loss by the chain rule."""
    y, (X, h1, h2) = forward(p, X)
    B = X.shape[0]
    gy = 2.0 * (y - t) / B                       # dL/dy
    g = {}
    g["W3"] = gy[None, :] @ h2
    g["b3"] = np.array([gy.sum()])
    gh2 = gy[:, None] * p["W3"]                  # [B, H]
    gz2 = gh2 * (1.0 - h2 * h2)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(axis=0)
    gh1 = gz2 @ p["W2"]
    gz1 = gh1 * (1.0 - h1 * h1)
    g["W1"] = gz1.T @ X
    g["b1"] = gz1.sum(axis=0)
    return g


def numerical_grad(p, X, t, h=1e-6):
    """Central differences of the loss, entry by entry (small networks only)."""
    g = {}
    for k in NAMES:
        gk = np.zeros_like(p[k])
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[k][idx]
            p[k][idx] = old + h
            lp = loss(p, X, t)
            p[k][idx] = old - h
            lm = loss(p, X, t)
            p[k][idx] = old
            gk[idx] = (lp - lm) / (2 * h)
        g[k] = gk
    return g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; state holds m, v per parameter and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
