"""Failure detection of the device-side waits, without a GPU fault: every
spin-wait of the cooperative kernels is bounded by GPU time and reports
WL_ERR_TIMEOUT instead of hanging. One CTA waits in the grid barrier for CTAs
that never arrive (a count nothing reaches); the wait gives up, the kernel
returns, and the same context then runs a normal computation."""
import time

import numpy as np
import pytest

import wlgen
from oracle import graph, walks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_barrier_completes_when_every_cta_arrives():
    from paper_2601_11338_gb300 import wl
    assert wl.wl_selftest_bounded_wait(0) == wl.WL_OK


def test_barrier_wait_expires_with_timeout_status_and_context_survives():
    from paper_2601_11338_gb300 import wl
    from paper_2601_11338_gb300.api import WalkLaplacian
    t0 = time.perf_counter()
    rc = wl.wl_selftest_bounded_wait(1)
    dt = time.perf_counter() - t0
    assert rc == wl.WL_ERR_TIMEOUT, rc
    assert 1.5 <= dt <= 30.0, dt  # the limit is 2 s of GPU time
    # the context is usable: a small walk-degree solve still matches the oracle
    g = wlgen.erdos_renyi(300, 6, 4)
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5, tol=1e-13)
    Df = w.degrees().cpu().numpy()
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    want = walks.walk_degrees(walks.phi_resolvent_closed(A, 1.0, w.info["alpha"]))
    w.close()
    assert np.linalg.norm(Df - want) <= 1e-10 * np.linalg.norm(want)
