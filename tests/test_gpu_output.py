"""GPU parity of the output options through the C ABI (pg_gather_ex):
extra first-vertex emitter samples (Section 4, "Handling direct light") and
the final gather (Fig. 2 caption), against the FP64 oracle.

Bars: final-gather neighbour tables bit-exact; FP32 images within 1e-5
relative (max_i |x_i - x_o,i| / max(|x_o,i|, 1e-3 mean|x_o|)).
"""
import numpy as np
import pytest
import torch

import oracle
import pgrec
from pgrec import synthetic

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).mean() + 1e-300)
    return float((np.abs(got - ref) / den).max())


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg

    return pg


SCENES = {
    "cube": pgrec.CUBE_CONST.with_(extra_direct=4),
    "cloud": pgrec.CLOUD128.with_(width=64, height=64, spp=4, extra_direct=3),
    "dense": pgrec.CLOUD256_DENSE.with_(grid_res=64, width=40, height=40, spp=2, iters=20, extra_direct=5),
}


class Case:
    pass


@pytest.fixture(scope="module", params=list(SCENES))
def case(request, pg):
    sc = SCENES[request.param]
    c = Case()
    c.sc = sc
    c.rec = rec = pgrec.trace(sc)
    c.ref = oracle.forward(rec, rec["first"], rec["bg"], sc.spp, sc.width, sc.height, sc.k, sc.iters)
    c.q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    c.Dx = oracle.extra_direct(rec, rec["first"], rec, sc.extra_direct)
    V = pg.Vertices.from_records(rec)
    c.graph = pg.pg_build_graph(V, sc.k)
    _, c.D = pg.pg_aggregate(c.graph, V, "f32")
    c.L = pg.pg_propagate(c.graph, torch.from_numpy(rec["L0"]).cuda(), sc.iters)
    c.first = torch.from_numpy(rec["first"]).cuda()
    c.bg = torch.from_numpy(rec["bg"]).cuda()
    c.extra = pg.extra_from_records(rec)
    return c


def _img(c, pg, **kw):
    sc = c.sc
    return pg.pg_gather_ex(c.graph, c.L, c.D, c.first, c.bg, sc.spp, sc.width, sc.height, **kw)


def test_plain_options_equal_pg_gather(case, pg):
    sc = case.sc
    a = pg.pg_gather(case.graph, case.L, case.D, case.first, case.bg, sc.spp, sc.width, sc.height)
    b = _img(case, pg)
    assert torch.equal(a, b)
    assert rel_err(b.cpu().numpy(), case.ref["image"]) <= FP32_TOL


def test_extra_direct_image(case, pg):
    sc, rec, ref = case.sc, case.rec, case.ref
    img = _img(case, pg, extra=case.extra).cpu().numpy()
    want = oracle.gather(rec, ref["nbr"], ref["A"], ref["L"], ref["D"], rec["first"], rec["bg"], sc.spp, sc.width,
                         sc.height, Dpath=case.Dx)
    assert rel_err(img, want) <= FP32_TOL
    # the extra samples change the output
    assert rel_err(img, ref["image"]) > 1e-3


@pytest.mark.parametrize("kfg", [1, 5, 8, 16, 32])
def test_final_gather(case, pg, kfg):
    sc, rec, ref = case.sc, case.rec, case.ref
    img, fg = _img(case, pg, final_gather_k=kfg, want_fg_nbr=True)
    vals, nb = oracle.final_gather(rec, case.q, ref["L"], rec["first"], rec["bg"], kfg, D=ref["D"])
    assert np.array_equal(fg.cpu().numpy(), nb)
    want = vals.reshape(sc.height, sc.width, sc.spp).mean(axis=2)
    assert rel_err(img.cpu().numpy(), want) <= FP32_TOL
    if kfg == sc.k:
        # kNN graph: the final gather's neighbourhoods are the graph's rows
        f = rec["first"]
        rows = case.graph.neighbors().cpu().numpy()[np.where(f >= 0, f, 0)]
        assert np.array_equal(nb[f >= 0], rows[f >= 0])


def test_final_gather_with_extra_direct(case, pg):
    sc, rec, ref = case.sc, case.rec, case.ref
    img = _img(case, pg, final_gather_k=16, extra=case.extra).cpu().numpy()
    vals, _ = oracle.final_gather(rec, case.q, ref["L"], rec["first"], rec["bg"], 16, Dpath=case.Dx)
    assert rel_err(img, vals.reshape(sc.height, sc.width, sc.spp).mean(axis=2)) <= FP32_TOL


@pytest.mark.parametrize("level", [7, 8])
def test_final_gather_first_ring_and_resume(pg, level):
    """On grids of level 7 or more the final gather's queries run the
    first-ring kernel; on the fine grid most of them are queued and resume
    at ring 2 from their saved lists. A graph of k = 4 puts every kfg below
    on the query path (no reuse of graph rows)."""
    sc = pgrec.CLOUD128.with_(width=40, height=40, spp=4, k=4, iters=10)
    rec = pgrec.trace(sc)
    V = pg.Vertices.from_records(rec)
    graph = pg.pg_build_graph(V, sc.k, grid_level=level)
    assert graph.info()["grid_level"] == level
    ref = oracle.forward(rec, rec["first"], rec["bg"], sc.spp, sc.width, sc.height, sc.k, sc.iters)
    assert np.array_equal(graph.neighbors().cpu().numpy(), ref["nbr"])
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    _, D = pg.pg_aggregate(graph, V, "f32")
    L = pg.pg_propagate(graph, torch.from_numpy(rec["L0"]).cuda(), sc.iters)
    first, bg = torch.from_numpy(rec["first"]).cuda(), torch.from_numpy(rec["bg"]).cuda()
    for kfg in (5, 16, 32):
        img, fg = pg.pg_gather_ex(graph, L, D, first, bg, sc.spp, sc.width, sc.height, final_gather_k=kfg,
                                  want_fg_nbr=True)
        vals, nb = oracle.final_gather(rec, q, ref["L"], rec["first"], rec["bg"], kfg, D=ref["D"])
        assert np.array_equal(fg.cpu().numpy(), nb), kfg
        assert rel_err(img.cpu().numpy(), vals.reshape(sc.height, sc.width, sc.spp).mean(axis=2)) <= FP32_TOL


def test_final_gather_on_cluster_graph(pg):
    """Cluster neighbourhoods in the iteration, a kNN final gather at output."""
    sc = pgrec.CLOUD128.with_(width=48, height=48, spp=4)
    rec = pgrec.trace(sc)
    V = pg.Vertices.from_records(rec)
    graph = pg.pg_build_graph(V, sc.k, cluster_size=sc.k, cluster_seed=11)
    nbr = graph.neighbors().cpu().numpy()
    lvl = graph.info()["grid_level"]
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    want_nbr, _ = oracle.cluster_graph(q, sc.k, sc.k, 11, lvl)
    assert np.array_equal(nbr, want_nbr)
    ref = oracle.forward(rec, rec["first"], rec["bg"], sc.spp, sc.width, sc.height, sc.k, sc.iters, nbr=want_nbr)
    _, D = pg.pg_aggregate(graph, V, "f32")
    L = pg.pg_propagate(graph, torch.from_numpy(rec["L0"]).cuda(), sc.iters)
    first, bg = torch.from_numpy(rec["first"]).cuda(), torch.from_numpy(rec["bg"]).cuda()
    img, fg = pg.pg_gather_ex(graph, L, D, first, bg, sc.spp, sc.width, sc.height, final_gather_k=16,
                              want_fg_nbr=True)
    vals, nb = oracle.final_gather(rec, q, ref["L"], rec["first"], rec["bg"], 16, D=ref["D"])
    assert np.array_equal(fg.cpu().numpy(), nb)
    assert rel_err(img.cpu().numpy(), vals.reshape(sc.height, sc.width, sc.spp).mean(axis=2)) <= FP32_TOL


def test_random_records_ties_and_short_paths(pg):
    """Random records on a coarse lattice (many equal distances), empty
    camera paths, fewer points than some k, random extra samples."""
    V = synthetic.random_records(2999, seed=5, n_paths=2 * 30 * 20)
    for c in ("px", "py", "pz"):
        V[c] = (np.round(V[c] * 12) / 12).astype(np.float32)
    X = synthetic.random_extra(2 * 30 * 20, 2, seed=6)
    k, iters, spp, w, h = 8, 5, 2, 30, 20
    ref = oracle.forward(V, V["first"], V["bg"], spp, w, h, k, iters)
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    Vd = pg.Vertices.from_records(V)
    graph = pg.pg_build_graph(Vd, k)
    _, D = pg.pg_aggregate(graph, Vd, "f32")
    L = pg.pg_propagate(graph, torch.from_numpy(V["L0"]).cuda(), iters)
    first, bg = torch.from_numpy(V["first"]).cuda(), torch.from_numpy(V["bg"]).cuda()
    extra = pg.extra_from_records(X)
    Dx = oracle.extra_direct(V, V["first"], X, 2)
    for kfg in (3, 16, 32):
        img, fg = pg.pg_gather_ex(graph, L, D, first, bg, spp, w, h, final_gather_k=kfg, extra=extra,
                                  want_fg_nbr=True)
        vals, nb = oracle.final_gather(V, q, ref["L"], V["first"], V["bg"], kfg, Dpath=Dx)
        assert np.array_equal(fg.cpu().numpy(), nb), kfg
        assert rel_err(img.cpu().numpy(), vals.reshape(h, w, spp).mean(axis=2)) <= FP32_TOL, kfg


def test_tiny_and_empty(pg):
    V3 = synthetic.random_records(3, seed=1, n_paths=2, max_len=3)
    Vd = pg.Vertices.from_records(V3)
    graph = pg.pg_build_graph(Vd, 8)
    _, D = pg.pg_aggregate(graph, Vd)
    L = pg.pg_propagate(graph, torch.from_numpy(V3["L0"]).cuda(), 2)
    ref = oracle.forward(V3, V3["first"], V3["bg"], 2, 1, 1, 8, 2)
    q = oracle.quantize(V3["px"], V3["py"], V3["pz"], (0, 0, 0), (1, 1, 1))
    first, bg = torch.from_numpy(V3["first"]).cuda(), torch.from_numpy(V3["bg"]).cuda()
    img, fg = pg.pg_gather_ex(graph, L, D, first, bg, 2, 1, 1, final_gather_k=8, want_fg_nbr=True)
    vals, nb = oracle.final_gather(V3, q, ref["L"], V3["first"], V3["bg"], 8, D=ref["D"])
    assert np.array_equal(fg.cpu().numpy(), nb)
    assert rel_err(img.cpu().numpy(), vals.reshape(1, 1, 2).mean(axis=2)) <= FP32_TOL
    # no vertices: the background only
    empty = {f: np.zeros(0, np.float32) for f in pgrec.F32_FIELDS}
    empty["e_delta"] = np.zeros(0, np.uint8)
    empty["succ"] = np.zeros(0, np.int32)
    Ve = pg.Vertices.from_records(empty)
    ge = pg.pg_build_graph(Ve, 8)
    _, De = pg.pg_aggregate(ge, Ve)
    Le = pg.pg_propagate(ge, torch.zeros(0, device="cuda"), 3)
    bg = torch.rand(12, device="cuda")
    X = synthetic.random_extra(12, 2, seed=1)
    img = pg.pg_gather_ex(ge, Le, De, torch.full((12,), -1, dtype=torch.int32, device="cuda"), bg, 2, 3, 2,
                          final_gather_k=4, extra=pg.extra_from_records(X))
    np.testing.assert_allclose(img.cpu().numpy(), bg.view(2, 3, 2).mean(2).cpu().numpy(), rtol=1e-6)


def test_bad_options_rejected(pg):
    V = synthetic.random_records(200, seed=3, n_paths=40)
    Vd = pg.Vertices.from_records(V)
    graph = pg.pg_build_graph(Vd, 8)
    _, D = pg.pg_aggregate(graph, Vd)
    L = pg.pg_propagate(graph, torch.from_numpy(V["L0"]).cuda(), 2)
    first, bg = torch.from_numpy(V["first"]).cuda(), torch.from_numpy(V["bg"]).cuda()
    args = (graph, L, D, first, bg, 1, 8, 5)
    with pytest.raises(pg.PgError) as e:
        pg.pg_gather_ex(*args, final_gather_k=33)
    assert e.value.status == 6
    with pytest.raises(pg.PgError) as e:
        pg.pg_gather_ex(*args, final_gather_k=-1)
    assert e.value.status == 1
    X = synthetic.random_extra(40, 2, seed=2)
    ex = pg.extra_from_records(X)
    ex0 = dict(ex, m=0)
    with pytest.raises(pg.PgError) as e:
        pg.pg_gather_ex(*args, extra=ex0)
    assert e.value.status == 1
    bad = dict(X, x_Le=X["x_Le"].copy())
    bad["x_Le"][3] = -1.0
    with pytest.raises(pg.PgError) as e:
        pg.pg_gather_ex(*args, extra=pg.extra_from_records(bad))
    assert e.value.status == 1
    bad = dict(X, x_ey=X["x_ey"].copy())
    bad["x_ey"][5] = np.inf
    with pytest.raises(pg.PgError) as e:
        pg.pg_gather_ex(*args, extra=pg.extra_from_records(bad))
    assert e.value.status == 4
    # the graph stays usable
    img = pg.pg_gather_ex(*args, extra=ex, final_gather_k=4)
    assert torch.isfinite(img).all()
