"""Large dense forward-scattering workload at full size, through the C ABI:
256^3 fBm medium (sigma_t max 60, albedo 0.999, HG g = 0.9), area light plus
environment, 1024 x 1024 pixels, 8 spp, depth 256 -> 158.7 M vertices and
2.3e9 swept entries (past 2^31, so every 64-bit index path is exercised);
k = 16, 16-bit weights (U16, the 16-bit format that meets 2e-3 per pixel at
albedo 0.999), 50 sweeps, forward plus adjoint.

The FP64 oracle checks, one by one: kNN rows by brute force, the direct terms
of sampled rows, and one U16 sweep of sampled rows, held to the rounding
bound of their 16-bit weights. Against the FP64 oracle's full-size image
(tests/golden/dense256_oracle_image.txt, the central 64 x 64 crop and every
32nd pixel, written by make_dense256_reference.py from oracle/ only): U16
and FP16 within 2e-3 per pixel; BF16's error is reported. Properties: the
residuals fall, and the reverse sweep from the stored transpose equals the
atomic scatter of the stored rows.
"""
import numpy as np
import pytest
import torch

import oracle
import pgrec

pytestmark = pytest.mark.gpu

SC = pgrec.CLOUD256_DENSE
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg

    class R:
        pass

    r = R()
    r.pg = pg
    r.rec = pgrec.trace(SC)
    r.Vt = {k: torch.from_numpy(np.ascontiguousarray(r.rec[k])).cuda() for k in pg.VERTEX_F32 + ("e_delta", "succ")}
    r.V = pg.Vertices(r.Vt)
    r.L0 = torch.from_numpy(r.rec["L0"]).cuda()
    r.first = torch.from_numpy(r.rec["first"]).cuda()
    r.bg = torch.from_numpy(r.rec["bg"]).cuda()
    r.graph = pg.pg_build_graph(r.V, SC.k)
    r.nbr = r.graph.neighbors().cpu().numpy()
    c, D = pg.pg_aggregate(r.graph, r.V, "u16")
    r.c, r.D = c.cpu().numpy(), D.cpu().numpy()
    r.Lp = pg.pg_propagate(r.graph, r.L0, SC.iters - 1).cpu().numpy()
    L, res, done = pg.pg_propagate(r.graph, r.L0, SC.iters, keep_history=True, want_residual=True)
    r.L, r.res, r.done = L.cpu().numpy(), res, done
    r.img = pg.pg_gather(r.graph, L, D, r.first, r.bg, SC.spp, SC.width, SC.height)
    r.info = r.graph.info()
    rng = np.random.default_rng(99)
    succ = r.rec["succ"]
    r.S = rng.choice(np.nonzero(succ >= 0)[0], 6, replace=False)
    yield r
    r.graph.close()


def test_size_past_int32(big):
    assert big.info["nnz_swept"] > 2 ** 31
    assert big.done == SC.iters
    assert np.all(np.diff(big.res) < 0) and big.res[-1] < 0.05 * big.res[0]


def test_knn_rows_bruteforce(big):
    q = oracle.quantize(big.rec["px"], big.rec["py"], big.rec["pz"], (0, 0, 0), (1, 1, 1))
    for s in big.S[:4]:
        d2 = ((q - q[s]) ** 2).sum(axis=1)
        d2[s] = np.iinfo(np.int64).max
        thr = np.partition(d2, SC.k - 2)[SC.k - 2]
        cand = np.nonzero(d2 <= thr)[0]
        cand = cand[np.lexsort((cand, d2[cand]))][:SC.k - 1]
        assert big.nbr[s, 0] == s
        assert np.array_equal(big.nbr[s, 1:], cand), s


def test_direct_terms_and_u16_sweep_rows(big):
    """Sampled rows s = succ(v): c_s and D_s within 1e-5 (they hold no 16-bit
    weight), and L_T[v] = w_s (sum_j W~_{s,j} L_{T-1}[j] / w_s + c_s) within
    the bound of the row's U16 payload: each weight is rounded to nearest
    on a 16-bit fixed-point grid of the row's largest weight, so it moves by
    at most 1/131070 of that weight (plus float32 rounding of the scale)."""
    succ = big.rec["succ"].astype(np.int64)
    rows = np.concatenate([big.S, succ[big.S]])
    ref = oracle.aggregate(big.rec, big.nbr, rows=rows)
    m = len(big.S)
    fl = 1e-3 * np.abs(big.c).mean()
    for name, got in (("c", big.c), ("D", big.D)):
        exp = ref[name]
        err = np.abs(got[rows] - exp) / np.maximum(np.abs(exp), fl)
        assert err.max() <= FP32_TOL, name
    s = succ[big.S]
    A = ref["A"][m:]
    w = big.rec["w_prop"].astype(np.float64)[s]
    nb = big.nbr[s]
    Lj = np.where(nb >= 0, big.Lp.astype(np.float64)[np.where(nb >= 0, nb, 0)], 0.0)
    Wt = w[:, None] * A
    expect = (Wt * Lj).sum(axis=1) + w * ref["c"][m:]
    bound = (1.0 / 131070 + 2.0 ** -22) * Wt.max(axis=1) * np.abs(Lj).sum(axis=1) + FP32_TOL * np.abs(expect) + 1e-30
    assert np.all(np.abs(big.L[big.S].astype(np.float64) - expect) <= bound)


def test_adjoint_modes_agree(big):
    """The reverse sweep from the stored transpose (64-bit column pointers
    here) against the atomic scatter of the stored rows: the same BF16
    operator through two code paths, equal to float32 summation order.

    A central difference of the forward map is no check at this workload: at
    albedo 0.999 the image's response to sigma_s is summed to ~1/(1 - a), so a
    step of 1e-2 is far outside the linear range, while at 1e-4 the BF16
    payloads of weights lying within a float32 rounding of a BF16 boundary
    flip between the two evaluations and swamp the difference (measured:
    -0.359 at h = 1e-2, -0.134 at h = 1e-4, against an adjoint of -0.301).
    The adjoint's central-difference checks run on the FP32 benchmark
    workload and the differentiation workload at full size.
    """
    pg = big.pg
    img0 = big.img.cpu().numpy().astype(np.float64)
    dI = torch.from_numpy((0.1 * img0).astype(np.float32).reshape(-1)).cuda()
    grads = []
    for mode in (0, 2):
        out = pg.pg_propagate_adjoint(big.graph, dI, big.first, SC.spp, SC.width, SC.height, want_g=False,
                                      recompute_weights=mode)
        grads.append(out["grad_sigma_s"].cpu().numpy().astype(np.float64))
    fl = 1e-3 * np.abs(grads[0]).max()
    assert (np.abs(grads[1] - grads[0]) / np.maximum(np.abs(grads[0]), fl)).max() <= 1e-4


def _dense_golden(big):
    import os
    import sys

    path = os.path.join(os.path.dirname(__file__), "golden", "dense256_oracle_image.txt")
    if not os.path.exists(path):
        pytest.skip("no stored FP64 oracle image of the dense workload")
    sys.path.insert(0, os.path.dirname(path))
    import make_dense256_reference as mod

    g = mod.load()
    if g["trace_sha256"] != mod.trace_checksum(big.rec):
        pytest.fail("the recorder's output differs from the one the stored oracle image was written from")
    return g


def _dense_image_error(img, g):
    y0, x0, crop = g["crop"]
    s_ = crop.shape[0]
    st, strided = g["stride"]
    floor = 1e-3 * np.abs(strided).mean()
    e1 = np.abs(img[y0:y0 + s_, x0:x0 + s_] - crop) / np.maximum(np.abs(crop), floor)
    e2 = np.abs(img[::st, ::st] - strided) / np.maximum(np.abs(strided), floor)
    return max(e1.max(), e2.max()), np.concatenate([e1.ravel(), e2.ravel()]).mean()


def test_u16_image_against_stored_oracle(big):
    """The 16-bit (U16) image of the full-size dense workload against the FP64
    oracle's, per pixel within 2e-3 on the crop and the strided grid."""
    g = _dense_golden(big)
    e_max, e_mean = _dense_image_error(big.img.cpu().numpy().astype(np.float64), g)
    print(f"\nu16 image vs FP64 oracle: max {e_max:.3e} mean {e_mean:.3e}")
    assert e_max <= 2e-3


@pytest.mark.parametrize("wdtype", ["f16", "bf16"])
def test_other_16bit_images_against_stored_oracle(big, wdtype):
    """FP16 within 2e-3 per pixel; BF16's error is measured and reported (its
    8-bit significand does not meet the bar at albedo 0.999)."""
    g = _dense_golden(big)
    pg = big.pg
    _, D = pg.pg_aggregate(big.graph, big.V, wdtype)
    L = pg.pg_propagate(big.graph, big.L0, SC.iters)
    img = pg.pg_gather(big.graph, L, D, big.first, big.bg, SC.spp, SC.width, SC.height)
    e_max, e_mean = _dense_image_error(img.cpu().numpy().astype(np.float64), g)
    print(f"\n{wdtype} image vs FP64 oracle: max {e_max:.3e} mean {e_mean:.3e}")
    if wdtype == "f16":
        assert e_max <= 2e-3
    del L, img


def test_fp32_sweep_rows(big):
    """FP32 weights on the same graph (the sweeps deal rows to the blocks in
    round-robin tiles at this size): one sweep of sampled rows against the
    oracle's row, L_T[v] = w_s (sum_j A+_{s,j} L_{T-1}[j] + c_s), within the
    FP32 tolerance; then the reverse sweeps in both schedules-independent
    modes agree. Runs last: it re-aggregates the module's graph."""
    pg = big.pg
    c, D = pg.pg_aggregate(big.graph, big.V, "f32")
    Lp = pg.pg_propagate(big.graph, big.L0, 9).cpu().numpy().astype(np.float64)
    L = pg.pg_propagate(big.graph, big.L0, 10, keep_history=True).cpu().numpy().astype(np.float64)
    succ = big.rec["succ"].astype(np.int64)
    s = succ[big.S]
    ref = oracle.aggregate(big.rec, big.nbr, rows=s)
    nb = big.nbr[s]
    Lj = np.where(nb >= 0, Lp[np.where(nb >= 0, nb, 0)], 0.0)
    w = big.rec["w_prop"].astype(np.float64)[s]
    expect = w * ((ref["A"] * Lj).sum(axis=1) + ref["c"])
    err = np.abs(L[big.S] - expect) / np.maximum(np.abs(expect), 1e-3 * np.abs(expect).mean())
    assert err.max() <= FP32_TOL
    img = pg.pg_gather(big.graph, torch.from_numpy(L.astype(np.float32)).cuda(), D, big.first, big.bg, SC.spp,
                       SC.width, SC.height)
    dI = (0.1 * img).reshape(-1).contiguous()
    g0 = pg.pg_propagate_adjoint(big.graph, dI, big.first, SC.spp, SC.width, SC.height, want_g=False,
                                 recompute_weights=0)["grad_sigma_s"].cpu().numpy().astype(np.float64)
    g2 = pg.pg_propagate_adjoint(big.graph, dI, big.first, SC.spp, SC.width, SC.height, want_g=False,
                                 recompute_weights=2)["grad_sigma_s"].cpu().numpy().astype(np.float64)
    fl = 1e-3 * np.abs(g0).max()
    assert (np.abs(g2 - g0) / np.maximum(np.abs(g0), fl)).max() <= 1e-4
