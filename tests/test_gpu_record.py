"""The GPU path recorder (pg_record_count / pg_record_fill through the C ABI)
against the host recorder: the same scene and seed give bit-identical
records (both evaluate the same double-precision operations in the same
order, with their own log and sin/cos), and the recorded path-tracer
estimate is what the oracle's K = 1 path graph recomputes from the records.
"""
import numpy as np
import pytest
import torch

import oracle
import pgrec

pytestmark = pytest.mark.gpu

SCENES = {
    "cube": pgrec.CUBE_CONST,
    "cloud": pgrec.CLOUD128.with_(width=64, height=64, spp=4, extra_direct=3),
    "grad": pgrec.CLOUD64_GRAD.with_(width=40, height=30, spp=3),
    "dense": pgrec.CLOUD256_DENSE.with_(grid_res=64, width=40, height=40, spp=2, extra_direct=2),
    "sun_only": pgrec.CLOUD128.with_(width=32, height=32, spp=2, sky_radiance=0.0, grid_res=48),
    "area_only": pgrec.CLOUD256_DENSE.with_(grid_res=32, width=32, height=24, spp=2, sky_radiance=0.0,
                                           max_depth=40, sigma_t_max=20.0),
}


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg

    return pg


def _record(pg, sc, albedo_grid=None):
    dens, alb = pgrec.medium(sc, albedo_grid)
    return pg.pg_record(sc, torch.from_numpy(dens).cuda(), torch.from_numpy(alb).cuda())


def _compare(gpu, host):
    assert gpu["n"] == host["n"] and gpu["n_paths"] == host["n_paths"]
    keys = list(pgrec.F32_FIELDS) + ["L0_f64", "e_delta", "succ", "voxel", "first", "bg", "pt_value"]
    if host.get("extra_direct", 0):
        keys += list(pgrec.EXTRA_F32) + ["x_delta"]
    for k in keys:
        g = gpu[k].cpu().numpy()
        assert g.dtype == host[k].dtype, k
        assert np.array_equal(g.view(np.uint8), np.ascontiguousarray(host[k]).view(np.uint8)), k


@pytest.mark.parametrize("name", list(SCENES))
def test_bit_identical_to_host_recorder(pg, name):
    sc = SCENES[name]
    _compare(_record(pg, sc), pgrec.trace(sc))


def test_albedo_grid_and_determinism(pg):
    sc = pgrec.CLOUD64_GRAD.with_(width=32, height=32, spp=2)
    rng = np.random.default_rng(4)
    ag = rng.uniform(0.9, 1.0, sc.grid_res ** 3).astype(np.float32)
    a = _record(pg, sc, ag)
    b = _record(pg, sc, ag)
    for k in ("px", "L0_f64", "succ", "pt_value"):
        assert torch.equal(a[k], b[k])
    _compare(a, pgrec.trace(sc, albedo_grid=ag))


def test_recorded_estimate_is_the_k1_path_graph(pg):
    """From the GPU's records alone: the oracle's K = 1 path graph (no
    neighbour edges) swept max_depth times from zero reproduces the recorded
    incoming indirect radiance, and its output the recorded path values."""
    sc = SCENES["grad"]
    g = _record(pg, sc)
    rec = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in g.items()}
    n = rec["n"]
    nbr = np.arange(n, dtype=np.int64)[:, None]
    agg = oracle.aggregate(rec, nbr)
    L, _, _ = oracle.propagate(rec, nbr, agg["A"], agg["c"], np.zeros(n), sc.max_depth)
    np.testing.assert_allclose(L, rec["L0_f64"], rtol=1e-12, atol=1e-300)
    vals = oracle.path_values(rec, nbr, agg["A"], L, agg["D"], rec["first"], rec["bg"])
    np.testing.assert_allclose(vals, rec["pt_value"], rtol=1e-12, atol=1e-15)


def test_full_size_bit_identical(pg):
    """The bench workload at full size (8.7 M vertices, 1 M paths)."""
    sc = pgrec.CLOUD128.with_(extra_direct=4)
    _compare(_record(pg, sc), pgrec.trace(sc))


def test_bad_scenes_rejected(pg):
    sc = pgrec.CUBE_CONST.with_(width=8, height=8, spp=1)
    dens, alb = pgrec.medium(sc)
    bad = dens.copy()
    bad[5] = -1.0
    with pytest.raises(pg.PgError) as e:
        pg.pg_record(sc, torch.from_numpy(bad).cuda(), torch.from_numpy(alb).cuda())
    assert e.value.status == 1
    bad = alb.copy()
    bad[3] = np.nan
    with pytest.raises(pg.PgError) as e:
        pg.pg_record(sc, torch.from_numpy(dens).cuda(), torch.from_numpy(bad).cuda())
    assert e.value.status == 1
    with pytest.raises(pg.PgError) as e:
        pg.pg_record(sc.with_(g=1.0), torch.from_numpy(dens).cuda(), torch.from_numpy(alb).cuda())
    assert e.value.status == 1
    # an empty medium: every camera ray leaves, no vertices
    z = np.zeros_like(dens)
    out = pg.pg_record(sc, torch.from_numpy(z).cuda(), torch.from_numpy(alb).cuda())
    assert out["n"] == 0 and bool((out["first"] == -1).all())
    _compare(out, pgrec.trace(sc.with_(sigma_t_max=0.0)))  # the host recorder on the same empty medium
