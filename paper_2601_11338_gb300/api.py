"""Convenience layer over the C ABI: keeps a graph on the GPU and returns
torch tensors. Marshalling only (device allocation of outputs, pointers,
status checks); all arithmetic runs in libwl.so."""
from __future__ import annotations

import numpy as np
import torch

from . import wl

VARIANTS = {"allwalk": wl.WL_ALLWALK, "nbt": wl.WL_NBT, "btdw": wl.WL_BTDW}
FUNCS = {"resolvent": wl.WL_F_RESOLVENT, "exp": wl.WL_F_EXP, "identity": wl.WL_F_IDENTITY}
PRECS = {"fp64": wl.WL_FP64, "refined": wl.WL_REFINED, "sketch": wl.WL_SKETCH}


def csr_to_device(row_ptr, col_idx, device="cuda"):
    rp = torch.as_tensor(np.asarray(row_ptr, dtype=np.int32)).to(device)
    ci = torch.as_tensor(np.asarray(col_idx, dtype=np.int32)).to(device)
    return rp, ci


class WalkLaplacian:
    """Handle on one graph and one walk Laplacian (variant, f, parameters)."""

    def __init__(self, row_ptr, col_idx, n, variant="allwalk", f="resolvent", alpha=0.0, alpha_rel=0.0,
                 mu=0.0, prec="fp64", tol=1e-12, max_iter=0, max_outer=0, outer_tol=0.0, device="cuda",
                 stream=None, reorder=1, beta=0.0, reorth=0, shift=0.0, gram=0):
        self.device = torch.device(device)
        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            self.row_ptr, self.col_idx = row_ptr, col_idx
        else:
            self.row_ptr, self.col_idx = csr_to_device(row_ptr, col_idx, self.device)
        self.n = int(n)
        self.nnz = int(self.col_idx.numel())
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        self.params = wl.make_params(f=FUNCS[f], alpha=alpha, alpha_rel=alpha_rel, beta=beta, mu=mu, prec=PRECS[prec],
                                     tol=tol, max_iter=max_iter, max_outer=max_outer, outer_tol=outer_tol,
                                     stream=s, reorder=reorder, reorth=reorth, shift=shift, gram=gram)
        self.build_stats = wl.wl_stats()
        self.h = wl.wl_build(self.row_ptr, self.col_idx, self.n, self.nnz, VARIANTS[variant], self.params,
                             self.build_stats)
        self.last = wl.wl_stats()

    def set(self, **kw):
        for k, v in kw.items():
            if k == "prec":
                v = PRECS[v]
            setattr(self.params, k, v)
        wl.wl_set_params(self.h, self.params)

    @property
    def info(self):
        return wl.wl_get_info(self.h).as_dict()

    def degrees(self, out=None, allow=()):
        Df = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        wl.wl_degrees(self.h, Df, self.last, allow)
        return Df

    def apply(self, V, out=None, allow=()):
        V = V.contiguous()
        k = V.shape[1]
        W = out if out is not None else torch.empty_like(V)
        wl.wl_apply(self.h, V, k, k, W, k, self.last, allow)
        return W

    def expmv(self, U0, taus, out=None, allow=()):
        U0 = U0.contiguous()
        k = U0.shape[1]
        taus = np.asarray(taus, dtype=np.float64)
        U = out if out is not None else torch.empty((len(taus), self.n, k), dtype=torch.float64,
                                                    device=U0.device)
        wl.wl_expmv(self.h, U0, k, k, taus, U, k, self.last, allow)
        return U

    def markov(self, P0, steps, out=None, allow=()):
        """Distributions of the chain P = D_f^{-1} phi after each of `steps` steps
        (columns of P0 are start distributions)."""
        P0 = P0.contiguous()
        k = P0.shape[1]
        steps = np.asarray(steps, dtype=np.int32)
        P = out if out is not None else torch.empty((len(steps), self.n, k), dtype=torch.float64,
                                                    device=P0.device)
        wl.wl_markov(self.h, P0, k, k, steps, P, k, self.last, allow)
        return P

    def return_prob(self, M, seed, ts, allow=()):
        """Estimates of tr(exp(-t L)) / n and their error estimates at each t."""
        return wl.wl_return_prob(self.h, M, seed, ts, self.last, allow)

    def trace(self, M, seed, omega_out=None):
        return wl.wl_trace(self.h, M, seed, omega_out, self.last)

    def warm_start(self, x0):
        wl.wl_set_warm_start(self.h, x0)

    def close(self):
        self.h.destroy()


def mlp_features(w: "WalkLaplacian"):
    """Node features (n x 4, FP32) and the analytic guess x_an (n, FP64) of a handle's graph."""
    F = torch.empty((w.n, 4), dtype=torch.float32, device=w.device)
    X = torch.empty(w.n, dtype=torch.float64, device=w.device)
    wl.wl_mlp_features(w.h, F, X)
    return F, X
