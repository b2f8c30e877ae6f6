"""Writes tests/golden/rmat14_trace.json: the exact trace of the all-walk
resolvent phi = (I - alpha A)^{-1}, alpha = 0.5 / lambda_max(A), on the seeded
R-MAT scale-14 graph (edge factor 16, a = .57, b = c = .19), from the dense
symmetric eigendecomposition of A: tr phi = sum_i 1 / (1 - alpha lambda_i).
Calls only the oracle and the input generators. Run: python tests/golden/make_rmat14_trace.py"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import wlgen  # noqa: E402
from oracle import graph  # noqa: E402

SEED = 20260300


def main():
    t = time.time()
    g = wlgen.rmat(14, 16, 0.57, 0.19, 0.19, seed=SEED)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    lam = np.linalg.eigvalsh(A)
    lmax = float(lam[-1])
    alpha = 0.5 / lmax
    tr = float(np.sum(1.0 / (1.0 - alpha * lam)))
    out = {"graph": "rmat", "scale": 14, "edge_factor": 16, "a": 0.57, "b": 0.19, "c": 0.19, "seed": SEED,
           "n": g.n, "nnz": g.nnz, "lambda_max": lmax, "alpha": alpha, "trace_allwalk_resolvent": tr,
           "how": "numpy.linalg.eigvalsh of the dense adjacency (oracle.graph.dense_adjacency)",
           "seconds": time.time() - t}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat14_trace.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
