"""pg_propagate_noalloc: propagation for callers that cannot allocate device
memory when they call it (for instance an application that gives the library
a fixed memory budget at start-up, or a per-frame loop that must not
allocate after set-up). The graph is built and aggregated at set-up, which
allocates; the checked call then keeps its scratch in a static device array.

Its result must equal pg_propagate's on the same graph, on two calls in a
row (the second call reuses the array the first one left behind).
"""
import ctypes

import numpy as np
import pytest
import torch

import pgrec

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).mean() + 1e-300)
    return float((np.abs(got - ref) / den).max())


@pytest.mark.parametrize("wdtype", ["f32", "f16"])
def test_noalloc_matches_pg_propagate(wdtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg
    from paper_2404_11894_gb300 import _lib

    lib = _lib.load()
    sc = pgrec.CLOUD128.with_(width=48, height=48, spp=4)
    rec = pgrec.trace(sc)
    V = pg.Vertices.from_records(rec)
    graph = pg.pg_build_graph(V, sc.k)
    pg.pg_aggregate(graph, V, wdtype)
    L0 = torch.from_numpy(rec["L0"]).cuda()
    ref = pg.pg_propagate(graph, L0, sc.iters)
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        st = lib.pg_propagate_noalloc(graph.handle, ctypes.c_void_p(L0.data_ptr()), sc.iters, 0.0,
                                      ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.pg_status_string(st)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    r = ref.cpu().numpy()
    for o in outs:
        assert np.isfinite(o).all()
        assert rel_err(o, r) <= FP32_TOL
    # sizes beyond the stated maximum are refused, not truncated
    big = lib.pg_propagate_noalloc(graph.handle, ctypes.c_void_p(L0.data_ptr()), 4097, 0.0,
                                   ctypes.c_void_p(ref.data_ptr()), stream)
    assert big == 6  # PG_ERR_UNSUPPORTED


def test_noalloc_early_stop_and_graph_change():
    """The array keeps whatever the last call left: a call with a stopping
    tolerance (which raises the device's stop flag) followed by calls without
    one, and a smaller graph after a larger one, must each still equal
    pg_propagate on the same graph and arguments."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg
    from paper_2404_11894_gb300 import _lib

    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    graphs = []
    for size in (64, 32):  # the larger graph first
        sc = pgrec.CLOUD128.with_(width=size, height=size, spp=4)
        rec = pgrec.trace(sc)
        V = pg.Vertices.from_records(rec)
        graph = pg.pg_build_graph(V, sc.k)
        pg.pg_aggregate(graph, V, "f32")
        graphs.append((sc, graph, torch.from_numpy(rec["L0"]).cuda()))
    for sc, graph, L0 in graphs:
        for tol in (0.05, 0.0, 0.05):
            ref, _, done = pg.pg_propagate(graph, L0, sc.iters, tol=tol, want_residual=True)
            if tol > 0:
                assert done < sc.iters  # the stop flag was raised on the device
            out = torch.full_like(ref, float("nan"))
            st = lib.pg_propagate_noalloc(graph.handle, ctypes.c_void_p(L0.data_ptr()), sc.iters, tol,
                                          ctypes.c_void_p(out.data_ptr()), stream)
            assert st == 0, lib.pg_status_string(st)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            assert np.isfinite(o).all()
            assert rel_err(o, ref.cpu().numpy()) <= FP32_TOL, (sc.width, tol)
