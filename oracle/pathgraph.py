"""FP64 CPU oracle for the volumetric path-graph hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it. It shares no code with the CUDA library.

It computes the path-graph estimator of "Rendering Participating Media Using
Path Graphs" (Hu et al.) step by step, in float64 with numpy, in the paper's
own form: the indirect radiance vector L+ indexed by vertex (Section 3.5,
Eq. rte-mff), the aggregation matrix A+ (Eq. ag-indirect / its matrix form),
the direct term A°L° (Eq. ag-direct), the propagation matrix P
(Eq. volume-propagation / rte-pg) and the per-path output (Section 4,
"Final output", "Handling direct light").

Readings where the paper is silent or garbled:
  * neighbourhoods are exact k-nearest-neighbour sets (self first, then the
    k-1 nearest others by squared integer distance, ties by smaller index) on
    21-bit quantised coordinates; the paper's clusters (Section 3.1) are the
    special case where every point's neighbourhood is its cluster;
  * the marginal density of a sample j (Eq. indirect-weight) is taken over the
    points that use j, R(j) = {s : j in N(s)}: with clusters every member's
    neighbourhood is the cluster, so R(j) is the cluster, and this is the
    reading that keeps, for any neighbour graph, the identity that a sample's
    MIS weights over the points aggregating it sum to one (which bounds the
    column sums of P A+ by the albedo, so the iteration contracts);
  * the "K p_E(omega_j)" inside the direct marginal (Eq. ag-direct, the
    definition of p_m after it) is read as K p_e of the same direction;
  * a delta-light emitter sample cannot be produced by phase sampling, so its
    balance-heuristic weight reduces to an average over the receiver's K
    emitter samples (K = |N(s)|); in the continuous-emitter and phase-sample
    marginals of Eq. ag-direct, K is |R(j)|, the number of emitter samples
    combined with the phase strategies of R(j);
  * Jacobi iteration (double-buffered), starting from the path tracer's
    estimate (Section 4, "Path graph solver"); sweep t=1 is the first
    aggregation + propagation;
  * "non-aggregated direct light" at output is the K=1 form of Eq. ag-direct.

Parity status of each function is stated in its docstring; the pins live in
``tests/test_oracle_pins.py``. The whole-pipeline bias against the exact RTE
solution is parity unpinned (the method is biased by design, Section 5).
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi
QBITS = 21
QMAX = (1 << QBITS) - 1


# --------------------------------------------------------------------------
# Graph build: quantisation and exact k nearest neighbours
# --------------------------------------------------------------------------
def quantize(px, py, pz, lo, hi):
    """21-bit integer coordinates of the vertices.

    q_a = min(2^21 - 1, max(0, floor((x_a - lo_a) * s))) with
    s = 2^21 / max_a(hi_a - lo_a). Every operation is one float32 operation
    with round-to-nearest (this is the single float32 step of the oracle, so
    that the integer coordinates, and with them the neighbour lists, are
    identical on every machine). Pinned by hand-computed cases.
    """
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    span = np.float32(max(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]))
    scale = np.float32(np.float32(1 << QBITS) / span)
    q = np.empty((len(px), 3), np.int64)
    for a, x in enumerate((px, py, pz)):
        t = (np.asarray(x, np.float32) - lo[a]) * scale  # float32 ops
        assert t.dtype == np.float32
        qa = np.floor(t).astype(np.int64)
        q[:, a] = np.clip(qa, 0, QMAX)
    return q


def knn_brute(q, k, r2_max=None):
    """Definition of the neighbourhood N(s), by brute force (O(n^2)).

    Row s: entry 0 is s itself; entries 1..k-1 are the other vertices with the
    smallest squared distance |q_s - q_j|^2 (exact int64), ties broken by the
    smaller index; with r2_max, entries farther than r2_max are dropped.
    Missing entries are -1. Pinned against a pure-Python loop.
    """
    n = len(q)
    nbr = -np.ones((n, k), np.int64)
    if n == 0 or k == 0:
        return nbr
    idx = np.arange(n)
    for s in range(n):
        d2 = ((q - q[s]) ** 2).sum(axis=1)
        order = np.lexsort((idx, d2))  # by d2, then index
        order = order[order != s][: k - 1]
        if r2_max is not None:
            order = order[d2[order] <= r2_max]
        nbr[s, 0] = s
        nbr[s, 1:1 + len(order)] = order
    return nbr


def knn(q, k, r2_max=None, workers=1, rows=None, tree=None):
    """Same neighbourhoods as :func:`knn_brute`, found with a k-d tree.

    scipy's cKDTree (a library kNN primitive) proposes candidate sets; each is
    re-ordered with exact int64 squared distances and index ties, and widened
    until the candidate set provably holds every point that can tie with the
    last kept entry. With ``rows`` only those query points are answered (row i
    of the result is point rows[i]'s neighbourhood among all points); ``tree``
    may pass a cKDTree already built over q (as float64) for repeated calls
    over row blocks. Pinned against :func:`knn_brute`.
    """
    from scipy.spatial import cKDTree

    n = len(q)
    qi = np.arange(n) if rows is None else np.asarray(rows, np.int64)
    nbr = -np.ones((len(qi), k), np.int64)
    if n == 0 or k == 0 or len(qi) == 0:
        return nbr
    nbr[:, 0] = qi
    if k == 1 or n == 1:
        return nbr
    if tree is None:
        tree = cKDTree(q.astype(np.float64))
    todo = np.arange(len(qi))
    kk = min(n, k + 8)
    while todo.size:
        pts = qi[todo]
        _, cand = tree.query(q[pts].astype(np.float64), k=kk, workers=workers)
        cand = np.asarray(cand, np.int64).reshape(len(todo), kk)
        d2 = ((q[cand] - q[pts][:, None, :]) ** 2).sum(axis=2)
        self_mask = cand == pts[:, None]
        d2s = np.where(self_mask, np.iinfo(np.int64).max, d2)
        # sort candidates by (d2, index), self last
        order = np.lexsort((cand, d2s), axis=1)
        cand_sorted = np.take_along_axis(cand, order, axis=1)
        d2_sorted = np.take_along_axis(d2s, order, axis=1)
        d2_far = d2.max(axis=1)  # every point outside the set is at least this far
        m = min(k - 1, n - 1)  # others wanted (all of them when n <= k-1)
        last = d2_sorted[:, m - 1]
        ok = (kk == n) | (last < d2_far)
        take = cand_sorted[ok, :m]
        dt = d2_sorted[ok, :m]
        take = np.where(dt == np.iinfo(np.int64).max, -1, take)  # never self
        if r2_max is not None:
            take = np.where(dt <= r2_max, take, -1)
        ncols = take.shape[1]
        nbr[todo[ok], 1:1 + ncols] = take
        todo = todo[~ok]
        kk = min(n, kk * 2)
    return nbr


# --------------------------------------------------------------------------
# Cluster neighbourhoods (Section 3.1, Section 4 "Path graph solver")
# --------------------------------------------------------------------------
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed, i):
    """Output i (0-based) of the SplitMix64 generator started from ``seed``:
    z = seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64) through the published
    finaliser (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31).
    Vectorised over i. Pinned by the generator's published first outputs."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(i, np.uint64) + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def morton_order(q, level):
    """Vertex indices ordered by the Morton code of their hash-grid cell at
    ``level`` (2^level cells per axis; cell = q >> (21 - level); bit b of
    x, y, z goes to bit 3b, 3b+1, 3b+2 of the code), ties by caller index."""
    cell = np.asarray(q, np.int64) >> (QBITS - level)
    key = np.zeros(len(cell), np.int64)
    for b in range(level):
        for a in range(3):
            key |= ((cell[:, a] >> b) & 1) << (3 * b + a)
    return np.lexsort((np.arange(len(cell)), key))


def nearest_centre(q, centres):
    """Index into ``centres`` of each vertex's nearest centre: smallest exact
    int64 squared distance, ties by the smaller caller index of the centre.
    A k-d tree (library kNN primitive) proposes candidates; each set is
    re-ordered exactly and widened until it provably holds every centre that
    ties with the nearest. Pinned against brute force."""
    from scipy.spatial import cKDTree

    q = np.asarray(q, np.int64)
    centres = np.asarray(centres, np.int64)
    m = len(centres)
    out = np.empty(len(q), np.int64)
    tree = cKDTree(q[centres].astype(np.float64))
    todo = np.arange(len(q))
    kk = min(m, 4)
    while todo.size:
        _, cand = tree.query(q[todo].astype(np.float64), k=kk)
        cand = np.asarray(cand, np.int64).reshape(len(todo), kk)
        d2 = ((q[centres[cand]] - q[todo][:, None, :]) ** 2).sum(axis=2)
        order = np.lexsort((centres[cand], d2), axis=1)
        best = np.take_along_axis(cand, order[:, :1], axis=1)[:, 0]
        dbest = np.take_along_axis(d2, order[:, :1], axis=1)[:, 0]
        ok = (kk == m) | (d2.max(axis=1) > dbest)
        out[todo[ok]] = best[ok]
        todo = todo[~ok]
        kk = min(m, kk * 2)
    return out


def nearest_centre_brute(q, centres):
    """Definition of :func:`nearest_centre` by brute force (O(n m))."""
    q = np.asarray(q, np.int64)
    centres = np.asarray(centres, np.int64)
    out = np.empty(len(q), np.int64)
    for v in range(len(q)):
        d2 = ((q[centres] - q[v]) ** 2).sum(axis=1)
        out[v] = np.lexsort((centres, d2))[0]
    return out


def cluster_graph(q, k, K, seed, level):
    """Neighbourhoods from the paper's disjoint clusters (Section 3.1: about
    N/K centres, every point joins the nearest one, large clusters are split
    until the sizes are even; Section 4: centres drawn at random, nearest-
    centre search on the hash grid), read as:
      1. vertex v is a centre iff splitmix64(seed, v) < floor((2^64 - 1) / K)
         (expected n/K centres); with none drawn, vertex 0 is the centre;
      2. every vertex joins its nearest centre (:func:`nearest_centre`);
      3. a cluster of S > k members is cut into P = ceil(S / k) parts: with
         its members in Morton order (:func:`morton_order` at ``level``) the
         i-th (0-based) goes to part floor(i P / S), so sizes differ by at
         most one and none exceeds k;
      4. N(s) = s, then the other members of s's part in Morton order, -1
         padded to width k.
    Returns (nbr, part) with part[v] an id shared by the members of a part.
    Pinned by the partition invariants, brute-force nearest centres and the
    generator's published outputs."""
    q = np.asarray(q, np.int64)
    n = len(q)
    nbr = -np.ones((n, k), np.int64)
    if n == 0:
        return nbr, np.zeros(0, np.int64)
    thr = np.uint64((2 ** 64 - 1) // K)
    centres = np.nonzero(splitmix64(seed, np.arange(n)) < thr)[0]
    if len(centres) == 0:
        centres = np.array([0])
    owner = nearest_centre(q, centres)            # index into centres
    rank = np.empty(n, np.int64)
    order = morton_order(q, level)
    rank[order] = np.arange(n)                    # Morton position of each vertex
    members = np.lexsort((rank, owner))           # by cluster, then Morton order
    bounds = np.flatnonzero(np.r_[True, owner[members][1:] != owner[members][:-1], True])
    part = np.empty(n, np.int64)
    next_id = 0
    for a, b in zip(bounds[:-1], bounds[1:]):
        mem = members[a:b]
        S = b - a
        P = -(-S // k)
        pidx = (np.arange(S) * P) // S
        for p in range(P):
            grp = mem[pidx == p]
            part[grp] = next_id
            next_id += 1
            for s in grp:
                others = grp[grp != s]
                nbr[s, 0] = s
                nbr[s, 1:1 + len(others)] = others
    return nbr, part


# --------------------------------------------------------------------------
# Henyey-Greenstein phase function (Eq. standard-RTE's rho)
# --------------------------------------------------------------------------
def hg(o, d, g):
    """rho(o, d) = (1 - g^2) / (4 pi (1 + g^2 - 2 g mu)^(3/2)), mu = -o.d.

    o: outgoing direction (toward the previous vertex / camera), d: direction
    the light arrives from; g > 0 scatters forward. Arrays broadcast over the
    leading axes; the last axis of o and d is xyz. Pinned by normalisation
    and the closed forms at mu = +-1.
    """
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    g = np.asarray(g, np.float64)
    mu = -(o * d).sum(axis=-1)
    den = 1.0 + g * g - 2.0 * g * mu
    return (1.0 - g * g) / (FOUR_PI * den ** 1.5)


def hg_dg(o, d, g):
    """d rho / d g of :func:`hg` (for the adjoint). Pinned by finite differences."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    g = np.asarray(g, np.float64)
    mu = -(o * d).sum(axis=-1)
    den = 1.0 + g * g - 2.0 * g * mu
    return (-2.0 * g) / (FOUR_PI * den ** 1.5) - 1.5 * (1.0 - g * g) * (2.0 * g - 2.0 * mu) / (FOUR_PI * den ** 2.5)


# --------------------------------------------------------------------------
# Vertex records
# --------------------------------------------------------------------------
def vertex_arrays(V):
    """float64 views of the recorded per-vertex quantities (caller order)."""
    f = lambda k: np.asarray(V[k], np.float64)  # noqa: E731
    return dict(
        o=np.stack([f("ox"), f("oy"), f("oz")], axis=1),
        d=np.stack([f("dx"), f("dy"), f("dz")], axis=1),
        e=np.stack([f("ex"), f("ey"), f("ez")], axis=1),
        g=f("g"), sigma_s=f("sigma_s"), sigma_t=f("sigma_t"), w=f("w_prop"),
        Le=f("Le"), pe_e=f("pe_e"), Lph=f("Lph"), pe_ph=f("pe_ph"),
        delta=np.asarray(V["e_delta"]).astype(bool),
        succ=np.asarray(V["succ"], np.int64),
    )


# --------------------------------------------------------------------------
# Aggregation (Section 3.5)
# --------------------------------------------------------------------------
def sample_marginals(V, nbr, cols=None, g=None, chunk=1 << 18):
    """Marginal densities of every sample j over the points that use it.

    R(j) = {r : j in N(r)}; K_j = |R(j)|;
      pm_d[j] = sum_{r in R(j)} rho_r(o_r, d_j)   (phase sample of j)
      pm_e[j] = sum_{r in R(j)} rho_r(o_r, e_j)   (emitter sample of j)
    (Eq. indirect-weight's p_m, and the phase part of Eq. ag-direct's).
    With ``cols`` only those samples' marginals are formed (the others are
    zero). The table is walked in blocks of ``chunk`` rows. Parity: pinned by
    the MIS column sums (each sample's weights over R(j) sum to one) and by
    the isotropic closed form.
    """
    X = vertex_arrays(V)
    if g is not None:
        X["g"] = np.asarray(g, np.float64)
    n = len(X["g"])
    want = None
    if cols is not None:
        want = np.zeros(n, bool)
        want[np.asarray(cols, np.int64)] = True
    pm_d = np.zeros(n)
    pm_e = np.zeros(n)
    K = np.zeros(n)
    for a in range(0, len(nbr), chunk):
        nb = nbr[a:a + chunk]
        mask = nb >= 0
        if want is not None:
            mask &= want[np.where(mask, nb, 0)]
        r_loc, i_idx = np.nonzero(mask)
        if len(r_loc) == 0:
            continue
        r = r_loc + a
        j = nb[r_loc, i_idx].astype(np.int64)
        top = int(j.max()) + 1
        pm_d[:top] += np.bincount(j, weights=hg(X["o"][r], X["d"][j], X["g"][r]), minlength=top)
        pm_e[:top] += np.bincount(j, weights=hg(X["o"][r], X["e"][j], X["g"][r]), minlength=top)
        K[:top] += np.bincount(j, minlength=top)
    return pm_d, pm_e, K


def aggregate(V, nbr, sigma_s=None, g=None, rows=None, marginals=None):
    """Aggregation weights of the rows s (all, or ``rows``) of the neighbour
    table ``nbr`` (all n rows: the marginals need every point that uses a
    sample).

    Returns a dict (all float64; rows in the order of ``rows``, else caller
    order):
      A   (m,k): A+_{s,j} = sigma_s(s) rho_s(o_s, d_j) / pm_d[j]
                 (Eq. ag-indirect, marginal of Eq. indirect-weight over R(j))
      Ae  (m,k): A°_{s,2j}: emitter sample of j (Eq. ag-direct, first sum),
                 sigma_s rho_s(o_s,e_j) / (pm_e[j] + K_j pe_e_j), or
                 sigma_s rho_s(o_s,e_j) / |N(s)| for a delta light
      Aph (m,k): A°_{s,2j+1}: phase sample of j (Eq. ag-direct, second sum),
                 sigma_s rho_s(o_s,d_j) / (pm_d[j] + K_j pe_ph_j)
      c   (m):   (A°L°)_s = sum_j Ae_{s,j} Le_j + Aph_{s,j} Lph_j
      D   (m):   the same with N(s) = {s} (non-aggregated direct, Section 4)
      pm_d, pm_e, Kj (n): the marginals of :func:`sample_marginals`
    Entries for missing neighbours (-1) are 0. ``sigma_s``/``g`` override the
    recorded per-vertex values (used by finite differences); ``marginals``
    passes (pm_d, pm_e, Kj) already formed by :func:`sample_marginals`.
    Parity: pinned by the MIS column sums (Eq. indirect-weight), the isotropic
    closed form, and the K=1 reduction to the path tracer.
    """
    X = vertex_arrays(V)
    if sigma_s is not None:
        X["sigma_s"] = np.asarray(sigma_s, np.float64)
    if g is not None:
        X["g"] = np.asarray(g, np.float64)
    recv = np.arange(len(nbr)) if rows is None else np.asarray(rows, np.int64)
    nb = nbr[recv]
    valid = nb >= 0
    j = np.where(valid, nb, 0)
    if marginals is None:
        marginals = sample_marginals(V, nbr, cols=None if rows is None else np.unique(j[valid]), g=g)
    pm_d, pm_e, Kj = marginals
    Ks = valid.sum(axis=1).astype(np.float64)[:, None]
    o_s, g_s, sig_s = X["o"][recv], X["g"][recv], X["sigma_s"][recv]
    rho_sd = hg(o_s[:, None, :], X["d"][j], g_s[:, None])
    rho_se = hg(o_s[:, None, :], X["e"][j], g_s[:, None])
    pd, pe, K = pm_d[j], pm_e[j], Kj[j]
    safe = lambda x: np.where(valid, x, 1.0)  # noqa: E731
    A = sig_s[:, None] * rho_sd / safe(pd)
    Ae_cont = sig_s[:, None] * rho_se / safe(pe + K * X["pe_e"][j])
    Ae_delta = sig_s[:, None] * rho_se / Ks
    Ae = np.where(X["delta"][j], Ae_delta, Ae_cont)
    Aph = sig_s[:, None] * rho_sd / safe(pd + K * X["pe_ph"][j])
    A, Ae, Aph = (np.where(valid, M, 0.0) for M in (A, Ae, Aph))
    out = dict(A=A, Ae=Ae, Aph=Aph, pm_d=pm_d, pm_e=pm_e, Kj=Kj, K=Ks[:, 0])
    out["c"] = (Ae * X["Le"][j] + Aph * X["Lph"][j]).sum(axis=1)
    # non-aggregated direct: K = 1, N(s) = {s}
    o, e, d, gg = X["o"][recv], X["e"][recv], X["d"][recv], X["g"][recv]
    rho_e = hg(o, e, gg)
    rho_d = hg(o, d, gg)
    Le, pe_, Lph, pph = X["Le"][recv], X["pe_e"][recv], X["Lph"][recv], X["pe_ph"][recv]
    De = np.where(X["delta"][recv], rho_e * Le, rho_e * Le / (rho_e + pe_))
    Dp = rho_d * Lph / (rho_d + pph)
    out["D"] = X["sigma_s"][recv] * (De + Dp)
    return out


# --------------------------------------------------------------------------
# Propagation (Eq. volume-propagation, Eq. rte-mff) and output
# --------------------------------------------------------------------------
def sweep(V, nbr, A, c, L):
    """One Jacobi sweep of L+ <- P (A+ L+ + A°L°).

    For a vertex v with successor s = succ(v):
    L+_v = (tau/p_t)_s * (sum_{j in N(s)} A+_{s,j} L+_j + c_s); 0 if v ends
    its path. (tau/p_t)_s is the weight of the segment from v to s.
    """
    succ = np.asarray(V["succ"], np.int64)
    w = np.asarray(V["w_prop"], np.float64)
    Lj = np.where(nbr >= 0, L[np.where(nbr >= 0, nbr, 0)], 0.0)
    Lbar = (A * Lj).sum(axis=1) + c              # scattered radiance at every s
    s = np.where(succ >= 0, succ, 0)
    return np.where(succ >= 0, w[s] * Lbar[s], 0.0)


def propagate(V, nbr, A, c, L0, iters, keep_history=False):
    """iters Jacobi sweeps from L0 (the path tracer's estimate, Section 4).

    Returns (L, history, residuals): history[t] = L after t sweeps
    (history[0] = L0 with path ends set to zero);
    residuals[t-1] = ||L_t - L_{t-1}||_2 / ||L_t||_2.
    Parity: pinned by the dense solve (I - P A+)^-1 P A°L° on tiny graphs,
    the isotropic geometric series, and the K=1 path-tracing fixed point.
    """
    # L+ is indexed by continuation edges (Section 3.5, the vector of incoming
    # indirect radiance "from all the incoming continuation edges"): a vertex
    # whose path ends has no such edge, so its entry is zero from the start.
    succ = np.asarray(V["succ"], np.int64)
    L = np.where(succ >= 0, np.asarray(L0, np.float64), 0.0)
    hist = [L.copy()] if keep_history else None
    res = []
    for _ in range(iters):
        Ln = sweep(V, nbr, A, c, L)
        num = np.sqrt(((Ln - L) ** 2).sum())
        den = np.sqrt((Ln ** 2).sum())
        res.append(num / den if den > 0 else 0.0)
        L = Ln
        if keep_history:
            hist.append(L.copy())
    return L, hist, np.array(res)


def path_values(V, nbr, A, L, D, first, bg, Dpath=None):
    """Radiance each path carries into the camera (Section 4, "Final output").

    For a path whose first vertex is f: (tau/p_t)_f * (sum_{j in N(f)} A+_{f,j} L+_j + D_f),
    with the non-aggregated direct D_f ("Handling direct light"); plus the
    background seen by a camera ray that left the medium (bg, 0 otherwise).
    ``Dpath`` (per path) replaces D_f, e.g. by :func:`extra_direct`.
    """
    first = np.asarray(first, np.int64)
    bg = np.asarray(bg, np.float64)
    w = np.asarray(V["w_prop"], np.float64)
    Lj = np.where(nbr >= 0, L[np.where(nbr >= 0, nbr, 0)], 0.0)
    f = np.where(first >= 0, first, 0)
    Lbar = (A * Lj).sum(axis=1)[f]
    Lbar = Lbar + (D[f] if Dpath is None else np.asarray(Dpath, np.float64))
    return bg + np.where(first >= 0, w[f] * Lbar, 0.0)


def gather(V, nbr, A, L, D, first, bg, spp, width, height, Dpath=None):
    """Pixel = mean of its spp path values (box filter, one pixel per path)."""
    vals = path_values(V, nbr, A, L, D, first, bg, Dpath)
    return vals.reshape(height, width, spp).mean(axis=2)


def extra_direct(V, first, X, M):
    """Direct light at each path's first vertex from M extra emitter samples
    (Section 4, "Handling direct light": a few extra emitter samples at the
    first bounce replace the non-aggregated direct light in the output).

    Reading: the M emitter samples and the path's own phase sample at f are
    combined by the balance heuristic, with M samples of the emitter strategy
    and one of the phase strategy:
      D^x_f = sigma_s(f) [ sum_m rho_f(o_f,e_m) Le_m / (M pe_m + rho_f(o_f,e_m))
                           + rho_f(o_f,d_f) Lph_f / (M pe_ph_f + rho_f(o_f,d_f)) ]
    where a delta-light sample m (which phase sampling cannot produce)
    contributes sigma_s rho_f(o_f,e_m) Le_m / M instead. With M = 1 and the
    path's own emitter sample this is D_f. X holds x_ex, x_ey, x_ez, x_Le,
    x_pe, x_delta (M per path, path p's at [p*M, (p+1)*M)). Returns one value
    per path (0 where the path has no vertex). Parity: pinned by the M = 1
    reduction to D and by the expectation under a closed-form light field.
    """
    P = len(first)
    first = np.asarray(first, np.int64)
    Xv = vertex_arrays(V)
    has = first >= 0
    f = np.where(has, first, 0)
    o, g = Xv["o"][f], Xv["g"][f]
    e = np.stack([np.asarray(X[c], np.float64).reshape(P, M) for c in ("x_ex", "x_ey", "x_ez")], axis=2)
    Le = np.asarray(X["x_Le"], np.float64).reshape(P, M)
    pe = np.asarray(X["x_pe"], np.float64).reshape(P, M)
    delta = np.asarray(X["x_delta"]).astype(bool).reshape(P, M)
    rho_e = hg(o[:, None, :], e, g[:, None])
    term = np.where(delta, rho_e * Le / M, rho_e * Le / (M * pe + rho_e))
    rho_d = hg(o, Xv["d"][f], g)
    ph = rho_d * Xv["Lph"][f] / (M * Xv["pe_ph"][f] + rho_d)
    return np.where(has, Xv["sigma_s"][f] * (term.sum(axis=1) + ph), 0.0)


def final_gather(V, q, L, first, bg, kfg, D=None, Dpath=None, chunk=None):
    """Per-path output through a final gather: one more aggregation, at the
    first vertices only, after the iteration (the optional final gather of
    the Fig. 2 caption, which decorrelates neighbouring pixels).

    Reading: path p with first vertex f aggregates over its own neighbourhood
    N_fg(f) = the kfg nearest vertices of f (same rule as the graph build:
    self first, then by squared quantised distance, ties by index), with the
    balance heuristic of f over the phase strategies of N_fg(f):
      A^fg_{f,j} = sigma_s(f) rho_f(o_f,d_j) / sum_{l in N_fg(f)} rho_l(o_l,d_j)
      val_p = bg_p + (tau/p_t)_f (sum_{j in N_fg(f)} A^fg_{f,j} L+_j + D_f)
    (val_p = bg_p without a vertex); ``Dpath`` (per path) replaces D_f.
    ``q``: quantised positions (:func:`quantize`). Returns (values per path,
    neighbour table of the paths (-1 rows for paths without a vertex)).
    Parity: pinned by the kfg = 1 reduction to the path tracer, the isotropic
    closed form, and the expectation under a closed-form radiance field.
    """
    first = np.asarray(first, np.int64)
    bg = np.asarray(bg, np.float64)
    has = first >= 0
    Xv = vertex_arrays(V)
    P = len(first)
    nb = -np.ones((P, kfg), np.int64)
    if has.any():
        nb[has] = knn(q, kfg, rows=first[has])
    L = np.asarray(L, np.float64)
    chunk = chunk or max(64, (1 << 20) // (kfg * kfg))  # paths per block: [p, l, j] tables stay ~100 MB
    f_all = np.where(has, first, 0)
    direct = np.asarray(D, np.float64)[f_all] if Dpath is None else np.asarray(Dpath, np.float64)
    indirect = np.zeros(P)
    for a in range(0, P, chunk):
        valid = nb[a:a + chunk] >= 0
        j = np.where(valid, nb[a:a + chunk], 0)
        f = f_all[a:a + chunk]
        d_j = Xv["d"][j]                                   # [p, j, xyz]
        # marginal of each sample j over the receiver's neighbourhood: [p, l, j]
        rho_lj = hg(Xv["o"][j][:, :, None, :], d_j[:, None, :, :], Xv["g"][j][:, :, None])
        pm = (rho_lj * valid[:, :, None]).sum(axis=1)
        rho_fj = hg(Xv["o"][f][:, None, :], d_j, Xv["g"][f][:, None])
        A = np.where(valid, Xv["sigma_s"][f][:, None] * rho_fj / np.where(valid, pm, 1.0), 0.0)
        indirect[a:a + chunk] = (A * np.where(valid, L[j], 0.0)).sum(axis=1)
    vals = bg + np.where(has, Xv["w"][f_all] * (indirect + direct), 0.0)
    return vals, nb


def forward(V, first, bg, spp, width, height, k, iters, lo=(0, 0, 0), hi=(1, 1, 1),
            r2_max=None, L0=None, nbr=None, keep_history=False, sigma_s=None, g=None):
    """Whole hot path: graph, aggregation, iters sweeps, image."""
    if nbr is None:
        q = quantize(V["px"], V["py"], V["pz"], lo, hi)
        nbr = knn(q, k, r2_max)
    agg = aggregate(V, nbr, sigma_s=sigma_s, g=g)
    if L0 is None:
        L0 = V["L0"]
    L, hist, res = propagate(V, nbr, agg["A"], agg["c"], L0, iters, keep_history)
    img = gather(V, nbr, agg["A"], L, agg["D"], first, bg, spp, width, height)
    return dict(nbr=nbr, L=L, history=hist, residuals=res, image=img, **agg)


def dense_fixed_point(V, nbr, A, c):
    """L+ = (I - P A+)^-1 P A°L° (Eq. rte-mff) by a dense LU solve, for tiny n.

    A+ and P are assembled as the paper's matrices: A+[s, nbr[s,j]] = A[s,j]
    (Eq. ag-indireect-mf) and P[v, succ(v)] = (tau/p_t)_{succ(v)} (Eq. rte-pg).
    """
    n = len(c)
    Ap = np.zeros((n, n))
    for s in range(n):
        for jj in range(nbr.shape[1]):
            if nbr[s, jj] >= 0:
                Ap[s, nbr[s, jj]] += A[s, jj]
    P = np.zeros((n, n))
    succ = np.asarray(V["succ"], np.int64)
    w = np.asarray(V["w_prop"], np.float64)
    for v in range(n):
        if succ[v] >= 0:
            P[v, succ[v]] = w[succ[v]]
    return np.linalg.solve(np.eye(n) - P @ Ap, P @ np.asarray(c, np.float64))


# --------------------------------------------------------------------------
# Adjoint: image-loss gradients through the fixed graph
# --------------------------------------------------------------------------
def adjoint(V, nbr, iters, L0, dI, first, bg, spp, width, height, voxel=None, n_vox=0, chunk=4096):
    """Reverse-mode derivative of the image w.r.t. per-vertex sigma_s and g.

    The differentiated map is theta -> image with theta = (sigma_s, g) per
    vertex; held fixed are positions, directions, light records, tau/p_t,
    L0 and the graph (weights are re-evaluated as functions of theta).
    ``dI`` is dLoss/dImage (height x width). Returns dict with grad_sigma_s,
    grad_g (per vertex) and, when ``voxel`` is given, grad_albedo per voxel
    (sigma_s = albedo * sigma_t, so d/dalbedo = sum over the voxel's vertices
    of sigma_t * d/dsigma_s).

    It is written as the chain rule through each weight formula: adjoints of
    A+, c and D first (reverse sweeps), then the explicit derivatives of the
    aggregation formulas. Parity: pinned by central finite differences of
    :func:`forward`.
    """
    X = vertex_arrays(V)
    n, k = nbr.shape
    agg = aggregate(V, nbr)
    A, c, D = agg["A"], agg["c"], agg["D"]
    L, hist, _ = propagate(V, nbr, A, c, L0, iters, keep_history=True)
    succ, w = X["succ"], X["w"]
    first = np.asarray(first, np.int64)
    valid = nbr >= 0
    j_idx = np.where(valid, nbr, 0)
    # path adjoints: nu_pi = dI[pixel]/spp
    nu_path = np.repeat(np.asarray(dI, np.float64).reshape(-1), spp) / spp
    hasf = first >= 0
    f = first[hasf]
    # adjoint of the per-row output weight w_f and of the quantities of row f
    gA = np.zeros((n, k))   # dLoss/dA+_{s,j}
    gc = np.zeros(n)        # dLoss/dc_s
    gD = np.zeros(n)        # dLoss/dD_s
    nu_row = np.zeros(n)
    np.add.at(nu_row, f, nu_path[hasf])
    gD += nu_row * w
    # lambda = dLoss/dL^(T) from the output
    lam = np.zeros(n)
    contrib = (nu_row * w)[:, None] * A
    np.add.at(lam, j_idx[valid], contrib[valid])
    gA += (nu_row * w)[:, None] * np.where(valid, hist[iters][j_idx], 0.0)
    # reverse sweeps t = iters .. 1: L^(t)_v = w_s (sum_j A_sj L^(t-1)_j + c_s)
    has_succ = succ >= 0
    v_rows = np.nonzero(has_succ)[0]
    s_rows = succ[v_rows]
    for t in range(iters, 0, -1):
        mu = np.zeros(n)                       # dLoss/d(scattered radiance at s)
        mu[s_rows] = lam[v_rows] * w[s_rows]
        gc += mu
        Lprev = hist[t - 1]
        gA += mu[:, None] * np.where(valid, Lprev[j_idx], 0.0)
        lam_prev = np.zeros(n)
        np.add.at(lam_prev, j_idx[valid], (mu[:, None] * A)[valid])
        lam = lam_prev
    # explicit derivatives of the aggregation formulas, per entry (s, j) with
    # j in N(s) (equivalently s in R(j)):
    #   A_sj  = sig_s rho_s(d_j) / pm_d[j]
    #   Ae_sj = sig_s rho_s(e_j) / me[j]  (delta: / |N(s)|),  me  = pm_e + K_j pe_e
    #   Aph_sj = sig_s rho_s(d_j) / mph[j],                    mph = pm_d + K_j pe_ph
    # g_s enters the numerators rho_s(o_s, .) of row s and, through
    # pm_d[j] and pm_e[j], the weights of every receiver of each j in N(s).
    grad_sig = np.zeros(n)
    grad_g = np.zeros(n)
    sig = X["sigma_s"]
    pm_d, pm_e, Kj = agg["pm_d"], agg["pm_e"], agg["Kj"]
    gpm_d = np.zeros(n)   # dLoss/dpm_d[j]
    gpm_e = np.zeros(n)   # dLoss/dpm_e[j]
    parts = []
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        nb = nbr[a:b]
        vm = nb >= 0
        j = np.where(vm, nb, 0)
        Ks = vm.sum(axis=1).astype(np.float64)[:, None]
        s_idx = np.arange(a, b)
        o_s, g_s = X["o"][s_idx], X["g"][s_idx]
        sg = sig[s_idx][:, None]
        d_j, e_j = X["d"][j], X["e"][j]
        rho_sd = hg(o_s[:, None, :], d_j, g_s[:, None])
        rho_se = hg(o_s[:, None, :], e_j, g_s[:, None])
        pd, pe, K = np.where(vm, pm_d[j], 1.0), np.where(vm, pm_e[j], 1.0), Kj[j]
        delta = X["delta"][j]
        Le, Lph = X["Le"][j], X["Lph"][j]
        me = np.where(vm, pe + K * X["pe_e"][j], 1.0)
        mph = np.where(vm, pd + K * X["pe_ph"][j], 1.0)
        gAc, gcc = gA[a:b], gc[a:b][:, None]
        # d/dsigma_s(s): every weight of row s is sigma_s(s) times a factor
        fA = np.where(vm, rho_sd / pd, 0.0)
        fe = np.where(vm, np.where(delta, rho_se / Ks, rho_se / me), 0.0)
        fph = np.where(vm, rho_sd / mph, 0.0)
        grad_sig[a:b] += (gAc * fA).sum(axis=1) + gcc[:, 0] * (fe * Le + fph * Lph).sum(axis=1)
        # adjoints of the marginals of the samples j (summed over receivers s)
        cd = np.where(vm, -sg * rho_sd * (gAc / pd ** 2 + gcc * Lph / mph ** 2), 0.0)
        ce = np.where(vm & ~delta, -sg * rho_se * gcc * Le / me ** 2, 0.0)
        np.add.at(gpm_d, j[vm], cd[vm])
        np.add.at(gpm_e, j[vm], ce[vm])
        # numerator factors of drho_s(o_s, d_j)/dg_s and drho_s(o_s, e_j)/dg_s
        nd = np.where(vm, sg * (gAc / pd + gcc * Lph / mph), 0.0)
        ne = np.where(vm, sg * gcc * Le * np.where(delta, 1.0 / Ks, 1.0 / me), 0.0)
        parts.append((a, b, nd, ne))
    for a, b, nd, ne in parts:
        nb = nbr[a:b]
        vm = nb >= 0
        j = np.where(vm, nb, 0)
        s_idx = np.arange(a, b)
        o_s, g_s = X["o"][s_idx], X["g"][s_idx]
        drho_sd = hg_dg(o_s[:, None, :], X["d"][j], g_s[:, None])
        drho_se = hg_dg(o_s[:, None, :], X["e"][j], g_s[:, None])
        tot = drho_sd * (nd + np.where(vm, gpm_d[j], 0.0)) + drho_se * (ne + np.where(vm, gpm_e[j], 0.0))
        grad_g[a:b] += np.where(vm, tot, 0.0).sum(axis=1)
    # D_s = sigma_s (De + Dp) with K = 1
    rho_e = hg(X["o"], X["e"], X["g"])
    rho_d = hg(X["o"], X["d"], X["g"])
    drho_e = hg_dg(X["o"], X["e"], X["g"])
    drho_d = hg_dg(X["o"], X["d"], X["g"])
    De = np.where(X["delta"], rho_e * X["Le"], rho_e * X["Le"] / (rho_e + X["pe_e"]))
    Dp = rho_d * X["Lph"] / (rho_d + X["pe_ph"])
    grad_sig += gD * (De + Dp)
    dDe = np.where(X["delta"], drho_e * X["Le"], drho_e * X["Le"] * X["pe_e"] / (rho_e + X["pe_e"]) ** 2)
    dDp = drho_d * X["Lph"] * X["pe_ph"] / (rho_d + X["pe_ph"]) ** 2
    grad_g += gD * sig * (dDe + dDp)
    out = dict(grad_sigma_s=grad_sig, grad_g=grad_g)
    if voxel is not None:
        ga = np.zeros(n_vox)
        np.add.at(ga, np.asarray(voxel, np.int64), X["sigma_t"] * grad_sig)
        out["grad_albedo"] = ga
    return out


def image_loss(img, target):
    """L = 1/2 sum_p (I_p - I*_p)^2 and its gradient dL/dI."""
    diff = np.asarray(img, np.float64) - np.asarray(target, np.float64)
    return 0.5 * float((diff ** 2).sum()), diff
