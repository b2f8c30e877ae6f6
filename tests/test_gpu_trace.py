"""XNysTrace through the C ABI against the oracle (Alg. 1, last step).

The sketch Omega is bit-exact (integer Philox words, FP64 Box-Muller on
both sides, bfloat16 rounding). The estimate is compared with the oracle's
literal leave-one-out estimate on the exact phi and the same Omega:

  FP64 form     Y by FP64 CG (tol 1e-13), FP64 Gram       1e-10 relative
  refined form  Y by the refined solve (tol 1e-12)         1e-8 relative
  sketch form   Y by FP32 CG (tol 1e-7), FP32 Gram on the  1e-5 relative
                CUDA cores (or, gram = 1, the two-term TF32
                Gram on the tensor cores) with FP32 sums per
                chunk

The sketch form's bound: Y carries a relative error of about kappa(M) 1e-7
(kappa(M) <= 3 at alpha = 0.5 / lambda_max) plus its FP32 rounding; the
Gram products are exact in the two-term TF32 split up to 2^-22 and are
summed in FP32 over chunks of about 4096 rows (at most a few 1e-6 relative);
the leave-one-out core multiplies these relative errors by about
cond(Omega^T phi Omega) (a few units here), so the estimate agrees to about
1e-5. The error estimate, a spread of nearly equal t_i, is compared within
1e-2 relative in the sketch form and 1e-6 in the others."""
import json
import os

import numpy as np
import pytest

import wlgen
from oracle import graph, philox, spectral, walks, xnys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rmat14_trace.json")


def WL(g, **kw):
    from paper_2601_11338_gb300.api import WalkLaplacian
    return WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, **kw)


@pytest.mark.parametrize("reorder", [0, 1])
@pytest.mark.parametrize("M", [64, 7, 2])
def test_sketch_is_bit_exact(M, reorder):
    g = wlgen.erdos_renyi(1000, 8, 3)
    w = WL(g, alpha_rel=0.5, reorder=reorder)
    om = torch.empty((g.n, M), dtype=torch.int16, device="cuda")
    w.trace(M, 12345 + M, om)
    got = om.cpu().numpy().view(np.uint16)
    _, want = philox.gaussian_sketch(g.n, M, 12345 + M)
    assert np.array_equal(got, want)


FORMS = {"fp64": (1e-13, 1e-10, 1e-6), "refined": (1e-12, 1e-8, 1e-6), "sketch": (1e-7, 1e-5, 1e-2)}


@pytest.mark.parametrize("prec", ["fp64", "refined", "sketch", "sketch_tc"])
@pytest.mark.parametrize("variant,mu,M,reorder", [("allwalk", 0.0, 64, 1), ("nbt", 1.0, 16, 0), ("btdw", 0.5, 7, 1)])
def test_estimate_matches_literal_leave_one_out(variant, mu, M, reorder, prec):
    gram = 1 if prec == "sketch_tc" else 0  # sketch_tc: the tensor-core Gram
    prec = "sketch" if gram else prec
    tol, etol, rtol = FORMS[prec]
    g = wlgen.erdos_renyi(700, 8, 4)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    w = WL(g, variant=variant, mu=mu, alpha_rel=0.5, tol=tol, prec=prec, reorder=reorder, gram=gram)
    alpha = w.info["alpha"]
    phi = walks.phi_resolvent_closed(A, mu, alpha)
    seed = 777 + M
    est, err = w.trace(M, seed)
    Om, _ = philox.gaussian_sketch(g.n, M, seed)
    e_o, r_o, _ = xnys.xnystrace(phi, Om)
    assert abs(est - e_o) <= etol * abs(e_o), (est, e_o)
    assert abs(err - r_o) <= rtol * r_o, (err, r_o)


def test_rmat14_estimate_against_exact_trace():
    """R-MAT scale 14, all-walk resolvent at alpha = 0.5 / lambda_max(A): the
    estimate lies within a few error estimates of the exact trace computed by
    the oracle's dense eigendecomposition (tests/golden/rmat14_trace.json)."""
    gold = json.load(open(GOLDEN))
    g = wlgen.rmat(gold["scale"], gold["edge_factor"], gold["a"], gold["b"], gold["c"], seed=gold["seed"])
    assert g.n == gold["n"] and g.nnz == gold["nnz"]
    w = WL(g, alpha=gold["alpha"], tol=1e-7, prec="sketch")
    ests = [w.trace(64, s) for s in (1, 2, 3)]
    tr = gold["trace_allwalk_resolvent"]
    for est, err in ests:
        assert abs(est - tr) <= 6 * err + 1e-6 * tr, (est, err, tr)
        assert err < 1e-2 * tr


@pytest.mark.parametrize("n,M,ldy", [(100_003, 64, 64), (4_097, 37, 64), (31, 64, 64), (0, 8, 8)])
def test_sketch_gram_tensor_cores(n, M, ldy):
    """The XNysTrace Gram [Omega Y]^T Y on the tensor cores (tcgen05, TF32
    with Y split in two terms) and on CUDA cores both match the FP64 product
    of the same inputs to FP32 accuracy; ragged row counts and sketch sizes."""
    from paper_2601_11338_gb300 import wl
    rng = np.random.default_rng(n + M)
    om32 = rng.normal(size=(n, M)).astype(np.float32)
    bits = (om32.view(np.uint32) >> 16).astype(np.uint16)  # BF16 patterns (truncated)
    om = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    Y = rng.normal(size=(n, ldy)).astype(np.float32)
    X = np.concatenate([om, Y[:, :M].astype(np.float64)], axis=1) if n else np.zeros((0, 2 * M))
    ref = np.zeros((128, 64))
    if n:
        P = X.T @ Y[:, :M].astype(np.float64)
        ref[:M, :M] = P[:M]
        ref[64:64 + M, :M] = P[M:]
    dom = torch.as_tensor(bits.view(np.int16) if n else np.zeros((1, M), np.int16), device="cuda")
    dY = torch.as_tensor(Y if n else np.zeros((1, ldy), np.float32), device="cuda")
    scale = np.abs(ref).max() if n else 1.0
    for tc in (0, 1):
        out = torch.full((128, 64), float("nan"), dtype=torch.float64, device="cuda")
        assert wl.wl_sketch_gram(dom, dY, n, M, ldy, tc, out) == wl.WL_OK
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 2e-6 * scale * max(1.0, np.sqrt(n) / 100), (tc, np.abs(got - ref).max())
