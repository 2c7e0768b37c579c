"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: closed
forms, the phase function's normalisation, brute force, the MIS identity
(the balance-heuristic weights of Eq. indirect-weight sum to one), the
geometric series of an infinite homogeneous medium, a dense solve of
Eq. rte-mff, the K = 1 reduction to the path tracer (Eqs. mc-indirect,
mc-pa), and finite differences for the adjoint.
"""
import os

import numpy as np
import pytest

import oracle
import pgrec
from pgrec import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- phase function
def _dirs_for_mu(mu):
    """o = +z and d with -o.d = mu."""
    mu = np.asarray(mu, np.float64)
    s = np.sqrt(np.clip(1 - mu * mu, 0, None))
    d = np.stack([s, np.zeros_like(mu), -mu], axis=-1)
    o = np.broadcast_to(np.array([0.0, 0.0, 1.0]), d.shape)
    return o, d


def test_hg_golden_special_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "hg_special_values.txt"))
    for g, mu, num, den in rows:
        o, d = _dirs_for_mu(np.array([mu]))
        got = oracle.hg(o, d, g)[0]
        assert got == pytest.approx(num / (den * np.pi), rel=1e-14), (g, mu)


@pytest.mark.parametrize("g", [0.0, 0.3, -0.3, 0.6, 0.8, 0.9, 0.99])
def test_hg_normalised(g):
    # int_{S^2} rho = 2 pi int_{-1}^{1} rho(mu) dmu, Gauss-Legendre on panels
    # refined toward the forward peak (mu = 1 for g > 0, -1 for g < 0)
    x, wq = np.polynomial.legendre.leggauss(64)
    edges = 1 - np.geomspace(2.0, 1e-9, 60)
    edges = np.concatenate([[-1.0], edges[edges > -1], [1.0]])
    edges = np.unique(edges if g >= 0 else -edges[::-1])
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        mu = 0.5 * (b - a) * x + 0.5 * (b + a)
        o, d = _dirs_for_mu(mu)
        total += 0.5 * (b - a) * (wq * oracle.hg(o, d, g)).sum()
    assert abs(2 * np.pi * total - 1.0) < 1e-10


def test_hg_forward_convention():
    # g > 0 scatters forward: light arriving from d continues along -d, so the
    # peak is at o = -d (mu = -o.d = 1)
    o = np.array([0.0, 0.0, 1.0])
    assert oracle.hg(o, -o, 0.8) > oracle.hg(o, o, 0.8)


def test_hg_dg_finite_difference():
    rng = np.random.default_rng(1)
    o, d = synthetic.unit_vectors(rng, 200).astype(np.float64), synthetic.unit_vectors(rng, 200).astype(np.float64)
    g = rng.uniform(-0.8, 0.95, 200)
    h = 1e-6
    fd = (oracle.hg(o, d, g + h) - oracle.hg(o, d, g - h)) / (2 * h)
    np.testing.assert_allclose(oracle.hg_dg(o, d, g), fd, rtol=1e-6, atol=1e-9)


# ---------------------------------------------------------------- quantisation
def test_quantize_hand_cases():
    x = np.array([0.0, 0.5, 1.0, -0.1, 0.25, np.float32(1 / 3), 1.5], np.float32)
    q = oracle.quantize(x, x, x, (0, 0, 0), (1, 1, 1))[:, 0]
    # 2^21 * 0.5 = 2^20; 1.0 -> 2^21 clamps to 2^21-1; negatives clamp to 0;
    # float32(1/3) = 0.3333333432674408 -> * 2^21 = 699050.6875 -> 699050
    assert q.tolist() == [0, 1 << 20, (1 << 21) - 1, 0, 1 << 19, 699050, (1 << 21) - 1]
    # non-cubic box: the largest extent sets one scale for all axes
    q2 = oracle.quantize(np.float32([1.0]), np.float32([1.0]), np.float32([0.5]), (0, 0, 0), (2, 1, 1))
    assert q2.tolist() == [[1 << 20, 1 << 20, 1 << 19]]


# ---------------------------------------------------------------- kNN
def _python_knn(q, k, r2_max=None):
    n = len(q)
    out = []
    for s in range(n):
        d2 = [int(((q[j] - q[s]) ** 2).sum()) for j in range(n)]
        others = sorted((j for j in range(n) if j != s), key=lambda j: (d2[j], j))[: k - 1]
        if r2_max is not None:
            others = [j for j in others if d2[j] <= r2_max]
        row = [s] + others
        out.append(row + [-1] * (k - len(row)))
    return np.array(out, np.int64)


def test_knn_brute_matches_python_loop():
    rng = np.random.default_rng(2)
    q = rng.integers(0, 4, size=(25, 3))  # many duplicates and ties
    for k in (1, 3, 8, 30):
        for r2 in (None, 2):
            np.testing.assert_array_equal(oracle.knn_brute(q, k, r2), _python_knn(q, k, r2))


@pytest.mark.parametrize("k", [1, 2, 5, 8, 16, 33])
def test_knn_tree_matches_brute(k):
    rng = np.random.default_rng(3 + k)
    for hi, n in ((6, 400), (1 << 21, 700), (3, 60)):
        q = rng.integers(0, hi, size=(n, 3))
        for r2 in (None, 4):
            np.testing.assert_array_equal(oracle.knn(q, k, r2), oracle.knn_brute(q, k, r2))


def test_knn_small_n():
    q = np.array([[0, 0, 0], [5, 0, 0], [1, 1, 1]])
    nbr = oracle.knn(q, 8)
    assert nbr.tolist()[0] == [0, 2, 1, -1, -1, -1, -1, -1]
    assert oracle.knn(q[:0], 4).shape == (0, 4)


# ---------------------------------------------------------------- aggregation
def _cluster_graph(**kw):
    V = synthetic.clustered_vertices(n_clusters=20, k=8, seed=4, **kw)
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, 8)
    # the neighbourhoods are the clusters
    assert (V["cluster"][nbr] == V["cluster"][:, None]).all()
    return V, nbr


def test_mis_weights_sum_to_one():
    """Eq. indirect-weight: for a fixed sample d_j the balance-heuristic
    weights over the K strategies of a cluster sum to one, so the column
    sums of A+ / sigma_s over the cluster are exactly 1."""
    V, nbr = _cluster_graph(random_g=True, random_sigma=True, pe_e=0.0, pe_ph=0.0, Lph=1.0)
    agg = oracle.aggregate(V, nbr)
    sig = V["sigma_s"].astype(np.float64)
    for name in ("A", "Ae", "Aph"):
        M = agg[name] / sig[:, None]
        for c in range(20):
            rows = np.nonzero(V["cluster"] == c)[0]
            # column j of row s is sample nbr[s, jj]; sum over rows s for each sample j
            col = {}
            for s in rows:
                for jj in range(8):
                    col[nbr[s, jj]] = col.get(nbr[s, jj], 0.0) + M[s, jj]
            np.testing.assert_allclose(list(col.values()), 1.0, rtol=1e-13)


def _knn_records(n=900, seed=12, k=8):
    """Random records on a kNN graph (neighbourhoods overlap and differ), with
    every emitter sample continuous and no emitter pdf mass, so the MIS sums
    of the direct weights reduce to the phase strategies alone."""
    V = synthetic.random_records(n, seed=seed)
    V["e_delta"] = np.zeros(n, np.uint8)
    V["pe_e"] = np.zeros(n, np.float32)
    V["pe_ph"] = np.zeros(n, np.float32)
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    return V, oracle.knn(q, k)


def knn_column_sums(M, nbr):
    """sum over the rows s that use sample j of M[s, slot of j]; and R(j)'s size."""
    valid = nbr >= 0
    n = nbr.shape[0]
    return (np.bincount(nbr[valid], weights=M[valid], minlength=n),
            np.bincount(nbr[valid], minlength=n))


def test_mis_weights_sum_to_one_on_knn_graphs():
    """Eq. indirect-weight on a neighbour graph that is not a set of clusters:
    sample j's balance-heuristic weights over the points that aggregate it
    (R(j), whose strategies form j's marginal) sum to one, so every column of
    A+ / sigma_s sums to exactly 1 and P A+ cannot grow a vector."""
    V, nbr = _knn_records()
    agg = oracle.aggregate(V, nbr)
    sig = V["sigma_s"].astype(np.float64)
    for name in ("A", "Ae", "Aph"):
        col, indeg = knn_column_sums(agg[name] / sig[:, None], nbr)
        assert indeg.min() >= 1 and indeg.max() > indeg.min()  # R(j) sizes differ
        np.testing.assert_allclose(col, 1.0, rtol=1e-13)
    # the column sums of P A+ (row v, sample j: w_succ(v) A+_{succ(v), j}) are
    # at most the largest albedo sigma_s / sigma_t
    X = oracle.vertex_arrays(V)
    a = X["sigma_s"] * X["w"]
    colP, _ = knn_column_sums(a[:, None] * agg["A"] / sig[:, None], nbr)
    assert colP.max() <= a.max() * (1 + 1e-13)


def test_weights_isotropic_closed_form_on_knn_graphs():
    """Isotropic rho = 1/(4 pi) on a kNN graph: A+_{s,j} = sigma_s / |R(j)|,
    Aph_{s,j} = sigma_s / (|R(j)| (1 + 4 pi pe_ph_j)), and a delta light's
    Ae_{s,j} = sigma_s / (4 pi |N(s)|)."""
    V, nbr = _knn_records(seed=13)
    V["g"] = np.zeros_like(V["g"])
    V["pe_ph"] = np.full_like(V["pe_ph"], 0.03)
    V["e_delta"] = np.ones_like(V["e_delta"])
    agg = oracle.aggregate(V, nbr)
    sig = V["sigma_s"].astype(np.float64)[:, None]
    _, indeg = knn_column_sums(np.ones(nbr.shape), nbr)
    Rj = indeg[nbr].astype(np.float64)
    pph = np.float64(np.float32(0.03))
    np.testing.assert_allclose(agg["A"], sig / Rj, rtol=1e-13)
    np.testing.assert_allclose(agg["Aph"], sig / (Rj * (1 + 4 * np.pi * pph)), rtol=1e-13)
    np.testing.assert_allclose(agg["Ae"], np.broadcast_to(sig / (4 * np.pi * nbr.shape[1]), nbr.shape), rtol=1e-13)


def test_sampled_rows_match_all_rows():
    """aggregate(rows=...) forms the same weights as the whole table (the
    marginals of a sampled row's samples still span every receiver)."""
    V, nbr = _knn_records(seed=14)
    full = oracle.aggregate(V, nbr)
    rows = np.array([0, 5, 17, 400, 899])
    part = oracle.aggregate(V, nbr, rows=rows)
    for name in ("A", "Ae", "Aph"):
        np.testing.assert_allclose(part[name], full[name][rows], rtol=1e-15)
    np.testing.assert_allclose(part["c"], full["c"][rows], rtol=1e-15)
    np.testing.assert_allclose(part["D"], full["D"][rows], rtol=1e-15)


def test_direct_weights_isotropic_closed_form():
    """Eq. ag-direct with isotropic rho = 1/(4 pi): the emitter sample's weight
    is sigma_s / (4 pi (K/(4 pi) + K pe)); a delta light's is sigma_s/(4 pi K)."""
    V, nbr = _cluster_graph(g=0.0, pe_e=0.05, pe_ph=0.02, Lph=1.0)
    agg = oracle.aggregate(V, nbr)
    sig = V["sigma_s"].astype(np.float64)[:, None]
    K = 8.0
    pe, pph = np.float64(np.float32(0.05)), np.float64(np.float32(0.02))
    full = lambda x: np.broadcast_to(x, agg["A"].shape)  # noqa: E731
    np.testing.assert_allclose(agg["Ae"], full(sig / (4 * np.pi) / (K / (4 * np.pi) + K * pe)), rtol=1e-13)
    np.testing.assert_allclose(agg["Aph"], full(sig / (4 * np.pi) / (K / (4 * np.pi) + K * pph)), rtol=1e-13)
    np.testing.assert_allclose(agg["A"], full(sig / K), rtol=1e-13)
    Vd, nbrd = _cluster_graph(g=0.0, delta=True)
    aggd = oracle.aggregate(Vd, nbrd)
    np.testing.assert_allclose(aggd["Ae"], full(Vd["sigma_s"].astype(np.float64)[:, None] / (4 * np.pi * K)),
                               rtol=1e-13)


# ---------------------------------------------------------------- iteration
def test_isotropic_infinite_medium_geometric_series():
    """Infinite homogeneous isotropic medium (cyclic paths, no path ends):
    every row of P A+ sums to the albedo a, and with a constant direct term
    b = a Le/(4 pi) the Jacobi iterate from zero is b (1 - a^t) / (1 - a)
    (the Neumann series of Eq. operator-RTE, scattering order n weighted a^n)."""
    a = 0.9
    V, nbr = _cluster_graph(g=0.0, albedo=a, sigma_t=3.0, delta=True, Le=2.0, cyclic=True)
    agg = oracle.aggregate(V, nbr)
    # the recorded float32 coefficients: a = sigma_s * (tau/p_t) = sigma_s / sigma_t
    af = np.float64(V["sigma_s"][0]) * np.float64(V["w_prop"][0])
    assert af == pytest.approx(a, rel=1e-6)
    b = af * 2.0 / (4 * np.pi)
    L = np.zeros(V["n"])
    for t in range(1, 40):
        L = oracle.sweep(V, nbr, agg["A"], agg["c"], L)
        np.testing.assert_allclose(L, b * (1 - af ** t) / (1 - af), rtol=1e-12)


@pytest.mark.parametrize("g,albedo", [(0.0, 0.9), (0.6, 0.6)])
def test_jacobi_matches_dense_solve(g, albedo):
    """Eq. rte-mff: the fixed point of the sweeps equals (I - P A+)^-1 P A°L°."""
    sc = pgrec.CUBE_CONST.with_(width=5, height=5, spp=1, g=g, albedo=albedo, sigma_t_max=2.0)
    rec = pgrec.trace(sc, nthreads=1)
    assert 8 <= rec["n"] <= 128, rec["n"]
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, 4)
    agg = oracle.aggregate(rec, nbr)
    Ld = oracle.dense_fixed_point(rec, nbr, agg["A"], agg["c"])
    L, _, res = oracle.propagate(rec, nbr, agg["A"], agg["c"], rec["L0"], 2000)
    np.testing.assert_allclose(L, Ld, rtol=1e-12, atol=1e-14 * np.abs(Ld).max())
    assert res[-1] < 1e-12


# ---------------------------------------------------------------- K = 1 reduction
SMALL_SCENES = [
    pgrec.CUBE_CONST.with_(width=24, height=24, spp=2),
    pgrec.CLOUD64_GRAD.with_(width=24, height=24, spp=2),
    pgrec.CLOUD256_DENSE.with_(grid_res=32, width=20, height=20, spp=1, max_depth=40, sigma_t_max=20.0),
]


@pytest.mark.parametrize("scene", SMALL_SCENES, ids=lambda s: s.name.split("_")[0])
def test_k1_reduces_to_path_tracing(scene):
    """With no neighbour edges (k = 1) the path graph is the path tracer
    (Eqs. mc-direct, mc-indirect, mc-pa): from zero, max_depth sweeps reach
    the tracer's own per-vertex estimate, and the output is its image."""
    rec = pgrec.trace(scene, nthreads=2)
    n = rec["n"]
    nbr = np.arange(n, dtype=np.int64)[:, None]
    agg = oracle.aggregate(rec, nbr)
    L, _, res = oracle.propagate(rec, nbr, agg["A"], agg["c"], np.zeros(n), scene.max_depth)
    np.testing.assert_allclose(L, rec["L0_f64"], rtol=1e-12, atol=1e-300)
    img = oracle.gather(rec, nbr, agg["A"], L, agg["D"], rec["first"], rec["bg"], scene.spp, scene.width, scene.height)
    np.testing.assert_allclose(img, rec["pt_image"], rtol=1e-12, atol=1e-15)
    # starting from the recorded float32 estimate the output stays on it
    L1, _, _ = oracle.propagate(rec, nbr, agg["A"], agg["c"], rec["L0"], 3)
    img1 = oracle.gather(rec, nbr, agg["A"], L1, agg["D"], rec["first"], rec["bg"], scene.spp, scene.width, scene.height)
    np.testing.assert_allclose(img1, rec["pt_image"], rtol=1e-6, atol=1e-9)


# ---------------------------------------------------------------- adjoint
def _loss(V, nbr, T, target, sc, sigma_s=None, g=None):
    out = oracle.forward(V, V["first"], V["bg"], sc.spp, sc.width, sc.height, sc.k, T, nbr=nbr,
                         sigma_s=sigma_s, g=g)
    return oracle.image_loss(out["image"], target)


def test_adjoint_matches_central_differences():
    sc = pgrec.CLOUD64_GRAD.with_(width=16, height=16, spp=2, k=8)
    rec = pgrec.trace(sc, nthreads=2)
    T = 6
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, sc.k)
    rng = np.random.default_rng(5)
    target = oracle.forward(rec, rec["first"], rec["bg"], sc.spp, sc.width, sc.height, sc.k, T, nbr=nbr,
                            sigma_s=rec["sigma_s"] * rng.uniform(0.9, 1.1, rec["n"]))["image"]
    base = oracle.forward(rec, rec["first"], rec["bg"], sc.spp, sc.width, sc.height, sc.k, T, nbr=nbr)
    _, dI = oracle.image_loss(base["image"], target)
    G = sc.grid_res
    adj = oracle.adjoint(rec, nbr, T, rec["L0"], dI, rec["first"], rec["bg"], sc.spp, sc.width, sc.height,
                         voxel=rec["voxel"], n_vox=G ** 3)
    sig0 = rec["sigma_s"].astype(np.float64)
    g0 = rec["g"].astype(np.float64)
    picks = rng.choice(rec["n"], 12, replace=False)
    for v in picks:
        h = 1e-4 * sig0[v]
        sp, sm = sig0.copy(), sig0.copy()
        sp[v] += h
        sm[v] -= h
        fd = (_loss(rec, nbr, T, target, sc, sigma_s=sp)[0] - _loss(rec, nbr, T, target, sc, sigma_s=sm)[0]) / (2 * h)
        assert adj["grad_sigma_s"][v] == pytest.approx(fd, rel=1e-6, abs=1e-12)
        h = 1e-5
        gp, gm = g0.copy(), g0.copy()
        gp[v] += h
        gm[v] -= h
        fd = (_loss(rec, nbr, T, target, sc, g=gp)[0] - _loss(rec, nbr, T, target, sc, g=gm)[0]) / (2 * h)
        assert adj["grad_g"][v] == pytest.approx(fd, rel=1e-5, abs=1e-11)
    # per-voxel albedo: sigma_s = albedo * sigma_t at every vertex of the voxel
    vox = np.unique(rec["voxel"])
    for vx in rng.choice(vox, 6, replace=False):
        m = rec["voxel"] == vx
        h = 1e-3
        st = rec["sigma_t"].astype(np.float64)
        sp, sm = sig0.copy(), sig0.copy()
        sp[m] += h * st[m]
        sm[m] -= h * st[m]
        fd = (_loss(rec, nbr, T, target, sc, sigma_s=sp)[0] - _loss(rec, nbr, T, target, sc, sigma_s=sm)[0]) / (2 * h)
        assert adj["grad_albedo"][vx] == pytest.approx(fd, rel=1e-6, abs=1e-12)


# ---------------------------------------------------------------- cluster neighbourhoods
def test_splitmix64_published_output():
    """The generator's first output from seed 0 is the published 0xE220A8397B1DCDAF;
    its top bits over many indices are uniform (the centre draw relies on it)."""
    assert int(oracle.splitmix64(0, 0)) == 0xE220A8397B1DCDAF
    top = oracle.splitmix64(12345, np.arange(1 << 16)) >> np.uint64(56)
    counts = np.bincount(top.astype(np.int64), minlength=256)
    assert counts.min() > 160 and counts.max() < 360  # mean 256, sd 16


def test_morton_order_matches_bit_interleave():
    rng = np.random.default_rng(8)
    q = rng.integers(0, 1 << 21, size=(300, 3))
    for level in (1, 3, 7):
        cell = q >> (21 - level)

        def code(c):
            out = 0
            for b in range(level):
                for a in range(3):
                    out |= ((int(c[a]) >> b) & 1) << (3 * b + a)
            return out

        keys = [code(c) for c in cell]
        want = sorted(range(len(q)), key=lambda i: (keys[i], i))
        np.testing.assert_array_equal(oracle.morton_order(q, level), want)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_nearest_centre_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    for hi, n in ((5, 300), (1 << 21, 500)):
        q = rng.integers(0, hi, size=(n, 3))  # the first case is full of ties
        centres = np.sort(rng.choice(n, max(1, n // 9), replace=False))
        np.testing.assert_array_equal(oracle.nearest_centre(q, centres), oracle.nearest_centre_brute(q, centres))


@pytest.mark.parametrize("K,k", [(4, 8), (8, 8), (16, 16), (40, 16)])
def test_cluster_graph_partition(K, k):
    """Section 3.1's clusters as neighbourhoods: a partition into parts of at
    most k points whose members share one neighbourhood (the part), each part
    inside the cluster of its points' nearest centre, the parts of one cluster
    even in size, about n/K centres."""
    rng = np.random.default_rng(K)
    n = 2000
    q = rng.integers(0, 1 << 21, size=(n, 3))
    level = 4
    nbr, part = oracle.cluster_graph(q, k, K, seed=77, level=level)
    thr = np.uint64((2 ** 64 - 1) // K)
    centres = np.nonzero(oracle.splitmix64(77, np.arange(n)) < thr)[0]
    assert abs(len(centres) - n / K) < 5 * np.sqrt(n / K)
    owner = oracle.nearest_centre_brute(q, centres)
    assert (nbr[:, 0] == np.arange(n)).all()
    for p in np.unique(part):
        mem = np.nonzero(part == p)[0]
        assert 1 <= len(mem) <= k
        assert len(np.unique(owner[mem])) == 1
        for s in mem:
            row = nbr[s][nbr[s] >= 0]
            assert sorted(row.tolist()) == sorted(mem.tolist())
            # others in Morton order
            rank = np.empty(n, np.int64)
            rank[oracle.morton_order(q, level)] = np.arange(n)
            assert np.all(np.diff(rank[row[1:]]) > 0)
    for c in np.unique(owner):
        sizes = np.bincount(part[owner == c])
        sizes = sizes[sizes > 0]
        assert sizes.max() - sizes.min() <= 1
        assert len(sizes) == -(-int((owner == c).sum()) // k)
