"""Pins of the oracle's output options: extra first-bounce emitter samples and
the final gather (Section 4, "Handling direct light"; the optional final
gather of the Fig. 2 caption).

Each test ties the oracle to something other than itself: the reduction to
the already-pinned direct term D and to the path tracer, an isotropic closed
form computed from brute-force neighbours, and Monte Carlo expectations under
light fields whose integrals against the Henyey-Greenstein phase function are
known in closed form (its mean cosine is g).
"""
import numpy as np
import pytest

import oracle
import pgrec
from pgrec import synthetic

from test_oracle_pins import SMALL_SCENES

FOUR_PI = 4.0 * np.pi


def _hg_sample(rng, o, g):
    """Directions d with density rho(o, d) (mu = -o.d), by rejection from the
    uniform sphere against the phase function's maximum."""
    n = len(o)
    out = np.empty((n, 3))
    todo = np.arange(n)
    while todo.size:
        d = synthetic.unit_vectors(rng, todo.size).astype(np.float64)
        gg = g[todo]
        mu = -(o[todo] * d).sum(axis=1)
        rho = (1 - gg * gg) / (FOUR_PI * (1 + gg * gg - 2 * gg * mu) ** 1.5)
        rmax = (1 - gg * gg) / (FOUR_PI * (1 - np.abs(gg)) ** 3)
        acc = rng.uniform(size=todo.size) * rmax < rho
        out[todo[acc]] = d[acc]
        todo = todo[~acc]
    return out


def test_hg_sampler_mean_cosine():
    """The test's own sampler reproduces the textbook mean cosine E[mu] = g."""
    rng = np.random.default_rng(5)
    n = 200_000
    o = np.tile([0.0, 0.0, 1.0], (n, 1))
    for g in (-0.4, 0.5, 0.85):
        d = _hg_sample(rng, o, np.full(n, g))
        mu = -d[:, 2]
        assert abs(mu.mean() - g) < 5 * mu.std() / np.sqrt(n)


def _records(n, o, g, sigma_s, d, Lph, pe_ph):
    V = {}
    for name, arr in (("o", o), ("d", d), ("e", d), ("p", np.zeros((n, 3)))):
        for a, ax in enumerate("xyz"):
            V[name + ax] = np.ascontiguousarray(arr[:, a])
    V.update(g=g, sigma_s=sigma_s, sigma_t=sigma_s, w_prop=np.ones(n), Le=np.zeros(n), pe_e=np.zeros(n),
             Lph=Lph, pe_ph=pe_ph, e_delta=np.zeros(n, np.uint8), succ=-np.ones(n, np.int32))
    return V


# ---------------------------------------------------------------- extra direct samples
@pytest.mark.parametrize("scene", SMALL_SCENES[:2], ids=lambda s: s.name.split("_")[0])
def test_extra_direct_single_own_sample_is_D(scene):
    """M = 1 with the path's own emitter sample as the extra one gives the
    non-aggregated direct term D_f (K = 1 form of Eq. ag-direct), and the
    output equals the path tracer's image."""
    rec = pgrec.trace(scene, nthreads=2)
    n = rec["n"]
    first = rec["first"].astype(np.int64)
    has = first >= 0
    f = np.where(has, first, 0)
    X = {"x_ex": rec["ex"][f], "x_ey": rec["ey"][f], "x_ez": rec["ez"][f], "x_Le": rec["Le"][f],
         "x_pe": rec["pe_e"][f], "x_delta": rec["e_delta"][f]}
    Dx = oracle.extra_direct(rec, first, X, 1)
    nbr = np.arange(n, dtype=np.int64)[:, None]
    agg = oracle.aggregate(rec, nbr)
    np.testing.assert_allclose(Dx[has], agg["D"][first[has]], rtol=1e-13, atol=1e-300)
    assert np.all(Dx[~has] == 0)
    img = oracle.gather(rec, nbr, agg["A"], rec["L0_f64"], agg["D"], rec["first"], rec["bg"], scene.spp,
                        scene.width, scene.height, Dpath=Dx)
    np.testing.assert_allclose(img, rec["pt_image"], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("M", [1, 3, 8])
def test_extra_direct_expectation(M):
    """Unbiased for any M: a sun (delta, picked with probability p_sun) and an
    environment Lenv(w) = 1 + a.w sampled uniformly; the phase sample sees
    the environment. E[D^x] = sigma_s (rho(o, sun) E + integral of rho Lenv)
    = sigma_s (rho(o, sun) E + 1 - g a.o)."""
    rng = np.random.default_rng(40 + M)
    P = 60_000
    p_sun, E = 0.3, 1.7
    a = np.array([0.3, -0.5, 0.4])
    sun = np.array([0.0, 0.6, 0.8])
    o = synthetic.unit_vectors(rng, P).astype(np.float64)
    g = rng.uniform(-0.3, 0.8, P)
    sigma_s = rng.uniform(0.5, 2.0, P)
    d = _hg_sample(rng, o, g)
    pe_c = (1 - p_sun) / FOUR_PI
    V = _records(P, o, g, sigma_s, d, 1 + d @ a, np.full(P, pe_c))
    pick = rng.uniform(size=(P, M)) < p_sun
    e = synthetic.unit_vectors(rng, P * M).astype(np.float64).reshape(P, M, 3)
    e = np.where(pick[:, :, None], sun, e)
    X = {"x_ex": e[:, :, 0].ravel(), "x_ey": e[:, :, 1].ravel(), "x_ez": e[:, :, 2].ravel(),
         "x_Le": np.where(pick, E / p_sun, 1 + e @ a).ravel(), "x_pe": np.where(pick, 0.0, pe_c).ravel(),
         "x_delta": pick.ravel().astype(np.uint8)}
    Dx = oracle.extra_direct(V, np.arange(P), X, M)
    mu_sun = -(o @ sun)
    rho_sun = (1 - g * g) / (FOUR_PI * (1 + g * g - 2 * g * mu_sun) ** 1.5)
    expect = sigma_s * (rho_sun * E + 1 - g * (o @ a))
    z = (Dx - expect).mean() / ((Dx - expect).std() / np.sqrt(P))
    assert abs(z) < 5, z


# ---------------------------------------------------------------- final gather
def test_knn_rows_match_brute():
    rng = np.random.default_rng(8)
    for hi, n in ((5, 300), (1 << 21, 500)):
        q = rng.integers(0, hi, size=(n, 3))
        rows = rng.choice(n, 40, replace=False)
        for k in (1, 4, 16, 33):
            np.testing.assert_array_equal(oracle.knn(q, k, rows=rows), oracle.knn_brute(q, k)[rows])


@pytest.mark.parametrize("scene", SMALL_SCENES, ids=lambda s: s.name.split("_")[0])
def test_final_gather_k1_reduces_to_path_tracing(scene):
    """With a one-point final-gather neighbourhood the output is the path
    tracer's image (Eqs. mc-direct, mc-indirect, mc-pa)."""
    rec = pgrec.trace(scene, nthreads=2)
    n = rec["n"]
    nbr = np.arange(n, dtype=np.int64)[:, None]
    agg = oracle.aggregate(rec, nbr)
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    vals, nb = oracle.final_gather(rec, q, rec["L0_f64"], rec["first"], rec["bg"], 1, D=agg["D"])
    np.testing.assert_allclose(vals, rec["pt_value"], rtol=1e-12, atol=1e-15)
    assert np.array_equal(nb[:, 0], np.where(rec["first"] >= 0, rec["first"], -1))


def test_final_gather_isotropic_closed_form():
    """g = 0: every phase density is 1/(4 pi), so the balance heuristic is a
    plain average over the brute-force neighbourhood:
    val = bg + w_f (sigma_s(f) mean_{j in N(f)} L_j + D_f)."""
    V = synthetic.random_records(3000, seed=21, n_paths=900)
    V["g"][:] = 0.0
    n = V["n"]
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    L = np.random.default_rng(3).uniform(0, 2, n)
    D = np.random.default_rng(4).uniform(0, 1, n)
    first = V["first"].astype(np.int64)
    has = first >= 0
    for k in (4, 16):
        vals, nb = oracle.final_gather(V, q, L, first, V["bg"], k, D=D)
        ref_nb = oracle.knn_brute(q, k)[first[has]]
        np.testing.assert_array_equal(nb[has], ref_nb)
        f = first[has]
        w = V["w_prop"].astype(np.float64)[f]
        ss = V["sigma_s"].astype(np.float64)[f]
        expect = V["bg"][has] + w * (ss * L[ref_nb].mean(axis=1) + D[f])
        np.testing.assert_allclose(vals[has], expect, rtol=1e-12)
        np.testing.assert_array_equal(vals[~has], V["bg"][~has].astype(np.float64))


def test_final_gather_expectation():
    """The final gather's balance heuristic is unbiased: groups of K points
    (each group is every member's K-neighbourhood), random o and g per point,
    phase samples d_l ~ rho_l and incoming radiance L(d) = 1 + a.d, so the
    receiver's estimate has expectation integral rho_f L = 1 - g_f a.o_f."""
    rng = np.random.default_rng(77)
    K, side = 8, 26
    G = side ** 3
    cid = np.repeat(np.arange(G), K)
    cen = (0.5 + np.stack([cid % side, (cid // side) % side, cid // side ** 2], axis=1)) / side
    pos = cen + 1e-4 * rng.uniform(-1, 1, size=(G * K, 3))
    n = G * K
    o = synthetic.unit_vectors(rng, n).astype(np.float64)
    g = rng.uniform(-0.4, 0.85, n)
    d = _hg_sample(rng, o, g)
    a = np.array([0.5, 0.2, -0.6])
    V = _records(n, o, g, np.ones(n), d, np.zeros(n), np.zeros(n))
    V["px"], V["py"], V["pz"] = (np.ascontiguousarray(pos[:, i]).astype(np.float32) for i in range(3))
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    first = np.arange(G) * K + rng.integers(0, K, G)
    vals, nb = oracle.final_gather(V, q, 1 + d @ a, first, np.zeros(G), K, D=np.zeros(n))
    assert np.array_equal(np.sort(nb, axis=1) // K, np.repeat(np.arange(G), K).reshape(G, K))
    expect = 1 - g[first] * (o[first] @ a)
    z = (vals - expect).mean() / ((vals - expect).std() / np.sqrt(G))
    assert abs(z) < 5, z


def test_extra_samples_leave_the_paths_unchanged():
    """The extra first-vertex samples come from a random stream of their own:
    every other record is identical with and without them."""
    sc = SMALL_SCENES[1]
    r0 = pgrec.trace(sc, nthreads=2)
    r1 = pgrec.trace(sc.with_(extra_direct=4), nthreads=2)
    for k, v in r0.items():
        if isinstance(v, np.ndarray):
            np.testing.assert_array_equal(r1[k], v, err_msg=k)
    P = r0["n_paths"]
    assert r1["x_Le"].shape == (4 * P,)
    none = np.repeat(r0["first"] < 0, 4)
    assert np.all(r1["x_Le"][none] == 0) and np.any(r1["x_Le"][~none] > 0)
    e = np.stack([r1["x_ex"], r1["x_ey"], r1["x_ez"]], axis=1).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(e, axis=1), 1.0, atol=1e-6)
