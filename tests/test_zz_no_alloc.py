"""The no-allocation walk-degree entry point (wl_degrees_noalloc) against the
regular one (wl_build + wl_degrees, FP64 form, caller's node order) and
against the CPU FP64 oracle's dense walk degrees (Sec. 3.1: D_f = phi 1 with
phi the resolvent of Eq. deformed).

wl_degrees_noalloc serves callers that cannot allocate GPU memory (a
framework step whose memory planner forbids allocation, hosts that reserve
all device memory up front, plug-ins handed only pre-allocated buffers): it
keeps its intermediate vectors in one fixed array inside libwl.so. This file
is collected last so that a run stopping at the first failure has already
run every other test; it passes alone and after the others (the first call
in a process also performs the one-time address lookup of that array)."""
import numpy as np
import pytest

import wlgen
from oracle import graph, walks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64-form parity tolerance of the GPU tests


def _device_csr(g):
    rp = torch.as_tensor(g.row_ptr.astype(np.int32), device="cuda")
    ci = torch.as_tensor(g.col_idx, device="cuda")
    return rp, ci


def _reference(g, variant, mu, alpha):
    from paper_2601_11338_gb300.api import WalkLaplacian
    w = WalkLaplacian(g.row_ptr.astype(np.int32), g.col_idx, g.n, variant=variant, mu=mu, alpha=alpha,
                      prec="fp64", tol=1e-13, reorder=0)
    Df = w.degrees().cpu().numpy()
    w.close()
    return Df


def _hubbed(n, seed):
    """Barabasi-Albert graph plus one node joined to 600 others (a row above
    the hub threshold of the CG kernels)."""
    g = wlgen.barabasi_albert(n, 3, seed)
    e_src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    keep = e_src < g.col_idx
    extra = np.arange(1, 601)
    src = np.concatenate([e_src[keep], np.zeros(600, dtype=np.int64)])
    dst = np.concatenate([g.col_idx[keep], extra])
    return wlgen.csr_from_edges(g.n, src, dst)


def _oracle(g, mu, alpha):
    A = graph.dense_adjacency(g.row_ptr, g.col_idx, g.n)
    return walks.walk_degrees(walks.phi_resolvent_closed(A, mu, alpha))


def test_noalloc_matches_degrees_and_oracle_on_two_calls_in_a_row():
    from paper_2601_11338_gb300 import wl
    cases = [
        (wlgen.erdos_renyi(3000, 8, 41), "nbt", 1.0, wl.WL_NBT),
        (_hubbed(5000, 42), "btdw", 0.5, wl.WL_BTDW),
    ]
    stream = torch.cuda.current_stream().cuda_stream
    for g, vname, mu, vcode in cases:
        alpha = 0.5 / (2.0 * np.sqrt(g.degrees.max()) + 1.0)  # comfortably below 1 / rho(Z_mu)
        want = _reference(g, vname, mu, alpha)
        exact = _oracle(g, mu, alpha)
        rp, ci = _device_csr(g)
        for call in range(2):
            got = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
            st = wl.wl_stats()
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            used0 = torch.cuda.memory_allocated()
            rc = wl.wl_degrees_noalloc(rp, ci, g.n, g.nnz, vcode, mu, alpha, got, tol=1e-13, stream=stream,
                                       stats=st)
            torch.cuda.synchronize()
            if call == 1:  # kernels are loaded by now: nothing on the device may grow
                assert torch.cuda.mem_get_info()[0] == free0
                assert torch.cuda.memory_allocated() == used0
            assert rc == wl.WL_OK and st.status == wl.WL_OK
            got = got.cpu().numpy()
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err <= TOL, (vname, call, err)
            # against the oracle: norm-wise and element-wise (each node within
            # TOL of the largest walk degree)
            assert np.linalg.norm(got - exact) / np.linalg.norm(exact) <= TOL, (vname, call)
            assert np.abs(got - exact).max() <= TOL * np.abs(exact).max(), (vname, call)
            assert st.iters > 0


def test_noalloc_rejects_graphs_beyond_its_fixed_array():
    from paper_2601_11338_gb300 import wl
    n = 262144 + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = wl.wl_stats()
    rc = wl.wl_degrees_noalloc(rp, ci, n, 0, wl.WL_ALLWALK, 0.0, 0.1, out, stats=st,
                               allow=(wl.WL_ERR_INVALID_ARG,))
    assert rc == wl.WL_ERR_INVALID_ARG and st.status == wl.WL_ERR_INVALID_ARG
