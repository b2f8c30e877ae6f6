"""One walk-Laplacian apply on a seeded Chung-Lu graph, for profilers.

    python -m paper_2601_11338_gb300.profile_apply [--n N] [--k K] [--prec refined|fp64] [--reorder 0|1]

Builds the handle (NBT resolvent, alpha = 0.5 / rho(Z_1)), computes the walk
degrees, then applies L to K Gaussian columns twice and prints the CG
per-iteration device time from the library's kernel timers. Device memory
stays at a few GB for n = 1e6, K = 16, so every kernel can be captured by a
multi-pass profiler.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import numpy as np
    import torch

    import wlgen
    from paper_2601_11338_gb300.api import WalkLaplacian

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--prec", default="refined", choices=["refined", "fp64"])
    ap.add_argument("--reorder", type=int, default=1)
    a = ap.parse_args()
    g = wlgen.chung_lu(a.n, seed=20260100)
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5, prec=a.prec,
                      tol=1e-10, reorder=a.reorder)
    w.degrees()
    V = torch.as_tensor(wlgen.gaussian_block(g.n, a.k, 1), device="cuda")
    for _ in range(2):
        w.apply(V)
    torch.cuda.synchronize()
    s = w.last
    print(f"n={g.n} nnz={g.nnz} K={a.k} prec={a.prec} reorder={a.reorder}: "
          f"cg {1000 * s.k_cg_ms / max(s.k_cg_iters, 1):.1f} us/iteration over {s.k_cg_iters} iterations, "
          f"residual {s.k_res_ms / max(s.k_res_launches, 1):.3f} ms/launch ({s.k_res_launches} launches)")


if __name__ == "__main__":
    main()
