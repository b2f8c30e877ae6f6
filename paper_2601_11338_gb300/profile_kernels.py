"""Small runs of the batched executor, the XNysTrace path and the warm-start
network, for profilers (each keeps a few GB on the device at most).

    python -m paper_2601_11338_gb300.profile_kernels batch   # 16 graphs x 5 mu, k = 32, refined
    python -m paper_2601_11338_gb300.profile_kernels trace   # R-MAT scale 18, M = 64
    python -m paper_2601_11338_gb300.profile_kernels mlp     # features + 20 training steps on 2e5 rows
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def batch():
    import numpy as np
    import torch

    import wlgen
    from paper_2601_11338_gb300 import wl
    gs = wlgen.batch_graphs(16, 1e3, 1e5, seed=20260200)
    n = sum(g.n for g in gs)
    graphs = [(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz) for g in gs]
    p = wl.make_params(f=wl.WL_F_RESOLVENT, alpha_rel=0.5, prec=wl.WL_REFINED, tol=1e-10,
                       stream=torch.cuda.current_stream().cuda_stream)
    b = wl.wl_batch_build(graphs, [1.0, 0.75, 0.5, 0.25, 0.0], p)
    V = torch.as_tensor(wlgen.gaussian_block(n, 32, 1), device="cuda")
    Df = torch.empty((5, n), dtype=torch.float64, device="cuda")
    W = torch.empty((5, n, 32), dtype=torch.float64, device="cuda")
    st = wl.wl_stats()
    for _ in range(2):
        wl.wl_batch_run(b, V, 32, Df, W, 0, st)
    torch.cuda.synchronize()
    print(f"batch: n={n} run {st.time_ms:.2f} ms, tile rows {wl.wl_batch_tile_rows(b, 32)}")


def trace():
    import numpy as np

    import wlgen
    from paper_2601_11338_gb300.api import WalkLaplacian
    g = wlgen.rmat(18, 16, 0.57, 0.19, 0.19, seed=20260318)
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="allwalk", alpha_rel=0.5,
                      prec="refined", tol=1e-7)
    for s in range(2):
        est, err = w.trace(64, s + 1)
    print(f"trace: n={g.n} nnz={g.nnz} estimate {est:.6g} +- {err:.3g}, {w.last.time_ms:.2f} ms")


def mlp():
    import numpy as np
    import torch

    import wlgen
    from paper_2601_11338_gb300 import warmstart, wl
    from paper_2601_11338_gb300.api import WalkLaplacian, mlp_features
    g = wlgen.chung_lu(200000, seed=20260500)
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5)
    F, X = mlp_features(w)
    D = w.degrees()
    T = torch.empty(g.n, dtype=torch.float32, device="cuda")
    wl.wl_mlp_targets(D, X, g.n, T)
    p = warmstart.initial_params(0)
    t0 = time.time()
    loss = wl.wl_mlp_train(p, F, T, g.n, 20, 0, 3e-3, 1)
    wl.wl_mlp_warm_start(w.h, p)
    torch.cuda.synchronize()
    print(f"mlp: rows={g.n} loss {loss:.4g} ({time.time() - t0:.2f} s)")


if __name__ == "__main__":
    {"batch": batch, "trace": trace, "mlp": mlp}[sys.argv[1]]()
