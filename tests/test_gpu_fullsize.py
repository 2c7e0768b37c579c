"""Parity at full size, through the same C-ABI calls and launch configuration
the benchmark times.

Benchmark workload (heterogeneous cloud: 8.7 M vertices, k = 16, 30 sweeps,
FP32). The FP64 oracle cannot run the whole workload inside a test, so it is
checked
  1. on outputs the oracle computes one by one: kNN rows by brute force,
     aggregation rows (c, D) of sampled vertices, one sweep of sampled rows
     from the GPU's previous iterate, and sampled pixels from the oracle's
     rows and the GPU's L+;
  2. against the oracle's full image stored in
     tests/golden/cloud128_oracle_image.txt (the central 64 x 64 crop and
     every 8th pixel; written by make_cloud128_reference.py, which calls only
     oracle/): FP32 within 1e-5, FP16 and BF16 weights within 2e-3 per pixel
     of the crop;
  3. on properties that hold at any size: the last sweep's residual, the graph
     counts, the adjoint against a central difference of the forward map
     along a random direction, and the three adjoint modes against each other.

Differentiation workload at full size (64^3 cloud, 128 x 128, 8 spp, 1.0 M
vertices, 20 sweeps): the per-voxel albedo gradient on 64 random occupied
voxels against the FP64 oracle's central differences (h = 1e-3, one voxel at
a time) and its adjoint, stored in tests/golden/cloud64_oracle_grad.txt.
"""
import numpy as np
import pytest
import torch

import oracle
import pgrec

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
W16_TOL = 2e-3
ADJ_TOL = 1e-3
SC = pgrec.CLOUD128


def rel_err(got, ref, floor=None):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    fl = 1e-3 * np.abs(ref).mean() if floor is None else floor
    den = np.maximum(np.abs(ref), fl + 1e-300)
    return np.abs(got - ref) / den


class Run:
    pass


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg

    return pg


def _tensor(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _forward(pg, r, wdtype="f32", sigma_s=None, iters=None, history=True):
    """Aggregate (with sigma_s overridden if given), propagate, gather."""
    V = r.V if sigma_s is None else pg.Vertices({**r.Vt, "sigma_s": _tensor(np.asarray(sigma_s, np.float32))})
    c, D = pg.pg_aggregate(r.graph, V, wdtype)
    L = pg.pg_propagate(r.graph, r.L0, r.sc.iters if iters is None else iters, keep_history=history)
    img = pg.pg_gather(r.graph, L, D, r.first, r.bg, r.sc.spp, r.sc.width, r.sc.height)
    torch.cuda.synchronize()
    return c, D, L, img


def _setup(pg, sc):
    r = Run()
    r.sc = sc
    r.rec = pgrec.trace(sc)
    r.Vt = {k: _tensor(r.rec[k]) for k in pg.VERTEX_F32 + ("e_delta", "succ")}
    r.V = pg.Vertices(r.Vt)
    r.graph = pg.pg_build_graph(r.V, sc.k)
    r.L0 = _tensor(r.rec["L0"])
    r.first = _tensor(r.rec["first"])
    r.bg = _tensor(r.rec["bg"])
    return r


@pytest.fixture(scope="module")
def full(pg):
    r = _setup(pg, SC)
    r.nbr = r.graph.neighbors().cpu().numpy()
    c, D, _, _ = _forward(pg, r)
    r.c, r.D = c.cpu().numpy(), D.cpu().numpy()
    r.Lp = pg.pg_propagate(r.graph, r.L0, SC.iters - 1).cpu().numpy()
    L, res, done = pg.pg_propagate(r.graph, r.L0, SC.iters, keep_history=True, want_residual=True)
    r.L, r.res, r.done = L.cpu().numpy(), res, done
    r.img = pg.pg_gather(r.graph, L, D, r.first, r.bg, SC.spp, SC.width, SC.height).cpu().numpy()
    r.info = r.graph.info()
    rng = np.random.default_rng(2024)
    n = r.rec["n"]
    r.q = oracle.quantize(r.rec["px"], r.rec["py"], r.rec["pz"], (0, 0, 0), (1, 1, 1))
    # sampled vertices: random ones, and the 16 with the farthest k-th neighbour
    # among 20000 random ones (the queries most likely to leave the first ring)
    pool = rng.choice(n, 20000, replace=False)
    last = r.nbr[pool, SC.k - 1]
    far = ((r.q[pool] - r.q[np.where(last >= 0, last, pool)]) ** 2).sum(axis=1)
    r.S = np.concatenate([rng.choice(n, 40, replace=False), pool[np.argsort(far)[-16:]]])
    yield r
    r.graph.close()


def _brute_row(q, s, k):
    """Neighbourhood of s by the definition: itself, then the k-1 others with
    the smallest exact squared distance, ties by smaller index."""
    d2 = ((q - q[s]) ** 2).sum(axis=1)
    d2[s] = np.iinfo(np.int64).max
    m = k - 1
    thr = np.partition(d2, m - 1)[m - 1]
    cand = np.nonzero(d2 <= thr)[0]
    cand = cand[np.lexsort((cand, d2[cand]))][:m]
    row = -np.ones(k, np.int64)
    row[0] = s
    row[1:1 + len(cand)] = cand
    return row


def test_knn_rows_bruteforce(full):
    for s in full.S:
        assert np.array_equal(full.nbr[s], _brute_row(full.q, s, SC.k)), s


def test_graph_counts(full):
    succ = full.rec["succ"]
    has_pred = np.zeros(full.rec["n"], bool)
    has_pred[succ[succ >= 0]] = True
    assert full.info["n_active"] == int(has_pred.sum())
    nb = full.nbr
    real = (nb >= 0) & (succ[np.where(nb >= 0, nb, 0)] >= 0)
    assert full.info["nnz_swept"] == int(real[has_pred].sum())


def test_aggregation_rows(full):
    S = full.S
    ref = oracle.aggregate(full.rec, full.nbr, rows=S)
    assert rel_err(full.c[S], ref["c"], floor=1e-3 * np.abs(full.c).mean()).max() <= FP32_TOL
    assert rel_err(full.D[S], ref["D"], floor=1e-3 * np.abs(full.D).mean()).max() <= FP32_TOL


def test_sweep_rows(full):
    """L_T[v] = w_s (sum_j A+_{s,j} L_{T-1}[j] + c_s), s = succ(v), for sampled v."""
    succ = full.rec["succ"].astype(np.int64)
    v = full.S[succ[full.S] >= 0]
    s = succ[v]
    ref = oracle.aggregate(full.rec, full.nbr, rows=s)
    nb = full.nbr[s]
    Lj = np.where(nb >= 0, full.Lp.astype(np.float64)[np.where(nb >= 0, nb, 0)], 0.0)
    w = full.rec["w_prop"].astype(np.float64)[s]
    expect = w * ((ref["A"] * Lj).sum(axis=1) + ref["c"])
    assert rel_err(full.L[v], expect, floor=1e-3 * np.abs(full.L).mean()).max() <= FP32_TOL
    # a path end carries nothing back
    ends = np.nonzero(succ < 0)[0][:1000]
    assert np.all(full.L[ends] == 0.0)


def test_last_residual(full):
    assert full.done == SC.iters
    L, Lp = full.L.astype(np.float64), full.Lp.astype(np.float64)
    r = np.sqrt(((L - Lp) ** 2).sum()) / np.sqrt((L ** 2).sum())
    assert full.res[-1] == pytest.approx(r, rel=1e-4)


def test_output_options_full_size(pg, full):
    """The output options at full size (1 M paths): final-gather neighbour
    tables equal the graph's rows for k_fg = k (kNN graph: their prefix) and
    brute force for sampled paths at k_fg = 24 (the exact search); the
    extra-sample image minus the plain one equals the oracle's
    (1/spp) sum_p (tau/p_t)_f (D^x_p - D_f) pixel by pixel."""
    from pgrec import synthetic

    rec, first_np = full.rec, full.rec["first"]
    L, D = _tensor(full.L), _tensor(full.D)
    has = first_np >= 0
    _, fg = pg.pg_gather_ex(full.graph, L, D, full.first, full.bg, SC.spp, SC.width, SC.height, final_gather_k=16,
                            want_fg_nbr=True)
    fg = fg.cpu().numpy()
    assert np.array_equal(fg[has], full.nbr[first_np[has]])
    assert np.all(fg[~has] == -1)
    _, fg24 = pg.pg_gather_ex(full.graph, L, D, full.first, full.bg, SC.spp, SC.width, SC.height, final_gather_k=24,
                              want_fg_nbr=True)
    fg24 = fg24.cpu().numpy()
    rng = np.random.default_rng(5)
    for p in rng.choice(np.nonzero(has)[0], 24, replace=False):
        assert np.array_equal(fg24[p], _brute_row(full.q, int(first_np[p]), 24)), p
    # extra first-vertex samples (random records, 2 per path)
    M = 2
    X = synthetic.random_extra(rec["n_paths"], M, seed=17)
    img_x = pg.pg_gather_ex(full.graph, L, D, full.first, full.bg, SC.spp, SC.width, SC.height,
                            extra=pg.extra_from_records(X)).cpu().numpy().astype(np.float64)
    Dx = oracle.extra_direct(rec, first_np, X, M)
    f = first_np[has].astype(np.int64)
    Df = oracle.aggregate(rec, np.arange(rec["n"], dtype=np.int64)[:, None], rows=f)["D"]
    w = rec["w_prop"].astype(np.float64)[f]
    delta = np.zeros(rec["n_paths"])
    delta[has] = w * (Dx[has] - Df)
    want = delta.reshape(SC.height, SC.width, SC.spp).mean(axis=2)
    got = img_x - full.img.astype(np.float64)
    scale = np.maximum(np.abs(full.img.astype(np.float64)), 1e-3 * np.abs(full.img).mean())
    assert (np.abs(got - want) / scale).max() <= FP32_TOL


def test_pixels_rows(full):
    rng = np.random.default_rng(7)
    pix = rng.choice(SC.width * SC.height, 24, replace=False)
    paths = (pix[:, None] * SC.spp + np.arange(SC.spp)[None, :]).ravel()
    f = full.rec["first"][paths].astype(np.int64)
    bg = full.rec["bg"][paths].astype(np.float64)
    live = f >= 0
    fr = f[live]
    ref = oracle.aggregate(full.rec, full.nbr, rows=fr)
    nb = full.nbr[fr]
    Lj = np.where(nb >= 0, full.L.astype(np.float64)[np.where(nb >= 0, nb, 0)], 0.0)
    w = full.rec["w_prop"].astype(np.float64)[fr]
    val = bg.copy()
    val[live] += w * ((ref["A"] * Lj).sum(axis=1) + ref["D"])
    expect = val.reshape(len(pix), SC.spp).mean(axis=1)
    got = full.img.reshape(-1)[pix]
    assert rel_err(got, expect, floor=1e-3 * np.abs(full.img).mean()).max() <= FP32_TOL


@pytest.fixture(scope="module")
def golden(full):
    import importlib.util
    import os

    p = os.path.join(os.path.dirname(__file__), "golden", "make_cloud128_reference.py")
    spec = importlib.util.spec_from_file_location("make_cloud128_reference", p)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    g = mod.load()
    if g["trace_sha256"] != mod.trace_checksum(full.rec):
        pytest.fail("the recorder's output differs from the one the stored oracle image was written from")
    return g


def _crop(img, g):
    y0, x0, crop = g["crop"]
    s = crop.shape[0]
    return img[y0:y0 + s, x0:x0 + s], crop


def test_image_against_stored_oracle(full, golden):
    floor = 1e-3 * np.abs(golden["stride"][1]).mean()
    got, ref = _crop(full.img, golden)
    assert rel_err(got, ref, floor).max() <= FP32_TOL
    st, strided = golden["stride"]
    assert rel_err(full.img[::st, ::st], strided, floor).max() <= FP32_TOL
    np.testing.assert_allclose(full.res, golden["residuals"], rtol=1e-3, atol=1e-7)


@pytest.mark.parametrize("wdtype", ["u16", "f16", "bf16"])
def test_16bit_crop_against_stored_oracle(pg, full, golden, wdtype):
    """Per-pixel relative error of the 64 x 64 crop against the FP64 oracle."""
    _, _, _, img = _forward(pg, full, wdtype=wdtype, history=False)
    got, ref = _crop(img.cpu().numpy(), golden)
    e = rel_err(got, ref, 1e-3 * np.abs(golden["stride"][1]).mean())
    print(f"\n{wdtype} crop error vs FP64 oracle: max {e.max():.3e} mean {e.mean():.3e}")
    assert e.max() <= W16_TOL


def _loss(img, target):
    d = np.asarray(img, np.float64) - target
    return 0.5 * float((d * d).sum())


def test_adjoint_direction_fd(pg, full):
    """<dLoss/dsigma_s, delta> against a central difference of the GPU forward
    map along a random relative perturbation delta of every sigma_s."""
    r = full
    sig = r.rec["sigma_s"].astype(np.float64)
    target = 0.9 * r.img.astype(np.float64)
    _, _, _, img = _forward(pg, r)
    dI = (img.cpu().numpy().astype(np.float64) - target).astype(np.float32).reshape(-1)
    out = pg.pg_propagate_adjoint(r.graph, _tensor(dI), r.first, SC.spp, SC.width, SC.height, want_g=False)
    gs = out["grad_sigma_s"].cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    delta = sig * rng.uniform(-1.0, 1.0, sig.shape)
    h = 1e-3
    lp = _loss(_forward(pg, r, sigma_s=sig + h * delta, history=False)[3].cpu().numpy(), target)
    lm = _loss(_forward(pg, r, sigma_s=sig - h * delta, history=False)[3].cpu().numpy(), target)
    fd = (lp - lm) / (2 * h)
    assert float(gs @ delta) == pytest.approx(fd, rel=ADJ_TOL)


def test_adjoint_modes_agree(pg, full):
    r = full
    _, _, _, img = _forward(pg, r)
    dI = (0.1 * img.cpu().numpy()).astype(np.float32).reshape(-1)
    outs = []
    for mode in (0, 2, 1):  # recompute (1) last: it runs after the stored weights are released
        if mode == 1:
            r.graph.release_weights()
        o = pg.pg_propagate_adjoint(r.graph, _tensor(dI), r.first, SC.spp, SC.width, SC.height, want_g=False,
                                    recompute_weights=mode)
        outs.append(o["grad_sigma_s"].cpu().numpy())
    ref = outs[0]
    fl = 1e-3 * np.abs(ref).max()
    for o in outs[1:]:
        assert rel_err(o, ref, fl).max() <= 1e-4


def test_voxel_albedo_central_differences_differentiation_workload(pg):
    """64^3 cloud at full size (128 x 128, 8 spp, 1.0 M vertices, 20 sweeps),
    L2 loss against a seeded target render (per-voxel albedo offsets in
    [-0.03, 0.03]): the per-voxel albedo gradient of pg_propagate_adjoint on
    64 random occupied voxels against the FP64 oracle's central differences
    (h = 1e-3, each voxel perturbed on its own) and the oracle's adjoint,
    both stored in tests/golden/cloud64_oracle_grad.txt by
    make_cloud64_reference.py (oracle/ only). Also the base and target images
    against the oracle's (every 4th pixel), and the chain rule through
    sigma_s."""
    import sys
    import os

    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_cloud128_reference as m128
    import make_cloud64_reference as m64

    gold = m64.load()
    sc = pgrec.CLOUD64_GRAD
    r = _setup(pg, sc)
    try:
        assert m128.trace_checksum(r.rec) == gold["trace_sha256"]  # the same traced inputs
        st = r.rec["sigma_t"].astype(np.float64)
        sig_tgt = (sc.albedo + m64.target_albedo_offsets(sc.grid_res)[r.rec["voxel"]]) * st
        tgt = _forward(pg, r, sigma_s=sig_tgt, history=False)[3].cpu().numpy().astype(np.float64)
        _, _, _, img = _forward(pg, r)
        img = img.cpu().numpy().astype(np.float64)
        s_ = gold["stride"]
        assert rel_err(img[::s_, ::s_], gold["image"]).max() <= FP32_TOL
        assert rel_err(tgt[::s_, ::s_], gold["target"]).max() <= FP32_TOL
        dI = (img - tgt).astype(np.float32).reshape(-1)
        nv = sc.grid_res ** 3
        out = pg.pg_propagate_adjoint(r.graph, _tensor(dI), r.first, sc.spp, sc.width, sc.height, want_g=False,
                                      voxel=_tensor(r.rec["voxel"]), sigma_t=_tensor(r.rec["sigma_t"]), n_vox=nv)
        ga = out["grad_albedo"].cpu().numpy().astype(np.float64)
        gs = out["grad_sigma_s"].cpu().numpy().astype(np.float64)
        pick = gold["voxels"]
        assert np.array_equal(pick, m64.pick_voxels(r.rec["voxel"]))
        fd, adj = gold["fd"], gold["adjoint"]
        floor = 1e-3 * np.abs(fd).max()
        assert rel_err(ga[pick], fd, floor).max() <= ADJ_TOL
        assert rel_err(ga[pick], adj, 1e-3 * np.abs(adj).max()).max() <= ADJ_TOL
        vox = r.rec["voxel"].astype(np.int64)
        chain = np.bincount(vox, weights=st * gs, minlength=nv)
        assert rel_err(ga[pick], chain[pick], 1e-3 * np.abs(chain[pick]).max()).max() <= 1e-4
    finally:
        r.graph.close()
