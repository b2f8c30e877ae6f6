"""Training of the warm-start network on walk degrees of generated graphs.

Marshalling only: features, solves, targets, training and inference run in
libwl.so (wl_mlp_features, wl_degrees, wl_mlp_targets, wl_mlp_train,
wl_mlp_warm_start). The initial weights are drawn here (Glorot-uniform,
seeded) and passed in.
"""
from __future__ import annotations

import numpy as np
import torch

from . import wl
from .api import WalkLaplacian, mlp_features

H = 64
N_IN = 4


def initial_params(seed: int = 0) -> np.ndarray:
    """Parameter vector (mean 0, std 1, Glorot-uniform weights, zero biases)."""
    rng = np.random.default_rng(seed)

    def glorot(fo, fi):
        lim = np.sqrt(6.0 / (fi + fo))
        return rng.uniform(-lim, lim, size=(fo, fi))

    parts = [np.zeros(N_IN), np.ones(N_IN), glorot(H, N_IN).ravel(), np.zeros(H), glorot(H, H).ravel(),
             np.zeros(H), glorot(1, H).ravel(), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == wl.wl_mlp_param_count()
    return p


def training_rows(graphs, variant="nbt", mu=0.0, alpha_rel=0.5, tol=1e-10):
    """Features and targets log(D_f / x_an) of every node of every graph (device tensors)."""
    Fs, Ts = [], []
    for g in graphs:
        w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant=variant, mu=mu, alpha_rel=alpha_rel,
                          prec="fp64", tol=tol)
        F, X = mlp_features(w)
        D = w.degrees()
        T = torch.empty(g.n, dtype=torch.float32, device=D.device)
        wl.wl_mlp_targets(D, X, g.n, T)
        Fs.append(F)
        Ts.append(T)
        w.close()
    return torch.cat(Fs).contiguous(), torch.cat(Ts).contiguous()


def train(graphs, variant="nbt", mu=0.0, alpha_rel=0.5, steps=2000, batch=0, lr=3e-3, seed=0):
    """Trained parameter vector (numpy float32) and its final training loss."""
    F, T = training_rows(graphs, variant, mu, alpha_rel)
    p = initial_params(seed)
    loss = wl.wl_mlp_train(p, F, T, F.shape[0], steps, batch, lr, 1,
                           torch.cuda.current_stream().cuda_stream)
    return p, loss
