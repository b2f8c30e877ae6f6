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


# ---------------------------------------------------------------- host-side fault injection (WL_FAULT)
def _small():
    g = wlgen.erdos_renyi(300, 6, 4)
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    return g, A


@pytest.fixture
def fault(monkeypatch):
    def set_mode(mode):
        monkeypatch.setenv("WL_FAULT", mode)
    yield set_mode
    monkeypatch.delenv("WL_FAULT", raising=False)


def _clean_solve_matches_oracle(g, A):
    from paper_2601_11338_gb300.api import WalkLaplacian
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5, tol=1e-13)
    Df = w.degrees().cpu().numpy()
    want = walks.walk_degrees(walks.phi_resolvent_closed(A, 1.0, w.info["alpha"]))
    w.close()
    return np.linalg.norm(Df - want) <= 1e-10 * np.linalg.norm(want)


@pytest.mark.parametrize("prec", ["fp64", "refined"])
@pytest.mark.parametrize("mode,status", [("nan", "WL_ERR_NONFINITE"), ("noconv", "WL_ERR_NO_CONVERGENCE")])
def test_injected_solver_faults_surface_as_status(fault, mode, status, prec):
    """A NaN in the starting residual and a one-iteration cap, made on the
    host, come back as the documented statuses; the next clean call on the
    same context is correct."""
    from paper_2601_11338_gb300 import wl
    from paper_2601_11338_gb300.api import WalkLaplacian
    g, A = _small()
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5, tol=1e-12, prec=prec)
    code = getattr(wl, status)
    fault(mode)
    w.degrees(allow=(code,))
    assert w.last.status == code
    fault("")
    w.close()
    assert _clean_solve_matches_oracle(g, A)


def test_injected_allocation_failure(fault):
    from paper_2601_11338_gb300 import wl
    g, A = _small()
    fault("alloc")
    rp = torch.as_tensor(g.row_ptr.astype(np.int32), device="cuda")
    ci = torch.as_tensor(g.col_idx, device="cuda")
    with pytest.raises(wl.WLError) as e:
        wl.wl_build(rp, ci, g.n, g.nnz, wl.WL_NBT, wl.make_params(alpha_rel=0.5))
    assert e.value.status == wl.WL_ERR_OOM
    fault("")
    assert _clean_solve_matches_oracle(g, A)


def test_injected_barrier_timeout(fault):
    """Every grid barrier starts in the gave-up state: the cooperative Lanczos
    step leaves at its first barrier and wl_expmv reports WL_ERR_TIMEOUT
    without waiting."""
    from paper_2601_11338_gb300 import wl
    from paper_2601_11338_gb300.api import WalkLaplacian
    g, A = _small()
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant="nbt", alpha_rel=0.5, tol=1e-12)
    U0 = torch.zeros((g.n, 1), dtype=torch.float64, device="cuda")
    U0[0, 0] = 1.0
    w.degrees()
    fault("timeout")
    t0 = time.perf_counter()
    w.expmv(U0, [1.0], allow=(wl.WL_ERR_TIMEOUT,))
    assert w.last.status == wl.WL_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 1.5  # no 2 s wait: the barrier had already given up
    fault("")
    w.close()
    assert _clean_solve_matches_oracle(g, A)


def test_injected_allocation_failure_in_the_batched_build(fault):
    """Every search thread of a batched build fails its first allocation: the
    threads leave the shared rounds as they fail, the build reports
    WL_ERR_OOM in bounded time, and a clean build afterwards is correct."""
    from oracle import spectral
    from paper_2601_11338_gb300 import wl
    gs = [wlgen.erdos_renyi(200 + 11 * i, 6.0, 500 + i) for i in range(24)]
    graphs = [(g.row_ptr.astype(np.int32), g.col_idx, g.n, g.nnz) for g in gs]
    p = wl.make_params(f=wl.WL_F_RESOLVENT, alpha_rel=0.5, prec=wl.WL_FP64, tol=1e-12,
                       stream=torch.cuda.current_stream().cuda_stream)
    fault("alloc")
    t0 = time.perf_counter()
    with pytest.raises(wl.WLError) as e:
        wl.wl_batch_build(graphs, [1.0, 0.5, 0.0], p)
    assert e.value.status == wl.WL_ERR_OOM
    assert time.perf_counter() - t0 < 30.0
    fault("")
    b = wl.wl_batch_build(graphs, [1.0, 0.5, 0.0], p)
    A = graph.dense_adjacency(gs[5].row_ptr, gs[5].col_idx, gs[5].n)
    rho = spectral.rho_companion(A, 1.0)
    assert abs(wl.wl_batch_info(b, 5, 0)["rho"] - rho) <= 1e-8 * rho
    b.destroy()
