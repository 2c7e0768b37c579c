"""Cluster neighbourhoods (the paper's disjoint clusters, Section 3.1 and
Section 4) on the GPU through the C ABI: neighbour lists bit-exact against the
FP64 oracle's cluster build, and the whole forward path on cluster graphs
against the oracle within 1e-5."""
import numpy as np
import pytest
import torch

import oracle
import pgrec
from pgrec import synthetic

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg

    return pg


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).mean() + 1e-300)
    return float((np.abs(got - ref) / den).max())


def _oracle_nbr(rec, k, K, seed, level):
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    nbr, _ = oracle.cluster_graph(q, k, K, seed, level)
    return nbr


@pytest.mark.parametrize("k,K,seed", [(8, 8, 1), (16, 16, 2), (16, 5, 3), (4, 40, 4)])
def test_cluster_neighbors_bit_exact_random(pg, k, K, seed):
    V = synthetic.random_records(6000, seed=seed)
    graph = pg.pg_build_graph(pg.Vertices.from_records(V), k, cluster_size=K, cluster_seed=seed)
    info = graph.info()
    want = _oracle_nbr(V, k, K, seed, info["grid_level"])
    assert np.array_equal(graph.neighbors().cpu().numpy(), want)
    assert info["clusters"] == len({tuple(sorted(r[r >= 0])) for r in want})


def test_cluster_neighbors_ties_and_duplicates(pg):
    """Lattice points: many equidistant centres and coincident positions."""
    rng = np.random.default_rng(9)
    n = 3000
    V = synthetic.random_records(n, seed=9)
    pos = (rng.integers(0, 10, size=(n, 3)) / 10.0).astype(np.float32)
    V["px"], V["py"], V["pz"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    for K in (3, 16):
        graph = pg.pg_build_graph(pg.Vertices.from_records(V), 8, cluster_size=K, cluster_seed=5, grid_level=3)
        want = _oracle_nbr(V, 8, K, 5, 3)
        assert np.array_equal(graph.neighbors().cpu().numpy(), want), K


def test_cluster_single_centre_fallback(pg):
    """K far above n: no centre is drawn, caller vertex 0 becomes the centre."""
    V = synthetic.random_records(40, seed=2, n_paths=40)
    graph = pg.pg_build_graph(pg.Vertices.from_records(V), 8, cluster_size=1 << 30, cluster_seed=1)
    want = _oracle_nbr(V, 8, 1 << 30, 1, graph.info()["grid_level"])
    assert np.array_equal(graph.neighbors().cpu().numpy(), want)


@pytest.mark.parametrize("scene", [pgrec.CUBE_CONST, pgrec.CLOUD128.with_(width=48, height=48, spp=4)],
                         ids=["cube", "cloud"])
def test_cluster_forward_parity(pg, scene):
    rec = pgrec.trace(scene)
    K, seed = scene.k, 11
    V = pg.Vertices.from_records(rec)
    graph = pg.pg_build_graph(V, scene.k, cluster_size=K, cluster_seed=seed)
    nbr = _oracle_nbr(rec, scene.k, K, seed, graph.info()["grid_level"])
    assert np.array_equal(graph.neighbors().cpu().numpy(), nbr)
    ref = oracle.forward(rec, rec["first"], rec["bg"], scene.spp, scene.width, scene.height, scene.k, scene.iters,
                         nbr=nbr)
    c, D = pg.pg_aggregate(graph, V, "f32")
    L, res, done = pg.pg_propagate(graph, torch.from_numpy(rec["L0"]).cuda(), scene.iters, want_residual=True)
    img = pg.pg_gather(graph, L, D, torch.from_numpy(rec["first"]).cuda(), torch.from_numpy(rec["bg"]).cuda(),
                       scene.spp, scene.width, scene.height)
    assert rel_err(c.cpu().numpy(), ref["c"]) <= FP32_TOL
    assert rel_err(D.cpu().numpy(), ref["D"]) <= FP32_TOL
    assert rel_err(L.cpu().numpy(), ref["L"]) <= FP32_TOL
    assert rel_err(img.cpu().numpy(), ref["image"]) <= FP32_TOL
    np.testing.assert_allclose(res, ref["residuals"], rtol=1e-3, atol=1e-7)
