"""Pins of the oracle's continuous-emitter and phase-sample weights of
Eq. ag-direct on kNN graphs, where a sample's user set R(j) = {s : j in N(s)}
and a receiver's neighbourhood N(s) differ in size.

On clusters the two counts coincide, so only a graph whose in-degrees vary
can tell which count multiplies the emitter pdf inside the marginal. Two
independent facts fix it:
  * a closed form: when every vertex has the same phase lobe (same outgoing
    direction and g), the marginal of K_j identical strategies is K_j rho, so
    each weight reduces to sigma_s rho / (K_j (rho + pe));
  * a Monte Carlo expectation: with identical lobes each sample's weights
    over the receivers that use it form a balance heuristic of K_j phase
    strategies and K_j emitter strategies, so the total direct term summed
    over all receivers is an unbiased estimate of n * integral(rho L) for a
    light field whose integral against the Henyey-Greenstein lobe is known in
    closed form (its mean cosine is g).
"""
import numpy as np
import pytest

import oracle
from pgrec import synthetic

from test_oracle_output_pins import _hg_sample

FOUR_PI = 4.0 * np.pi


def _identical_lobe_records(n, seed, g, o_dir=(0.3, -0.2, 0.93)):
    """kNN-graph records (random positions, k = 8) in which every vertex
    shares one outgoing direction and one g; continuous emitter samples only."""
    V = synthetic.random_records(n, seed=seed)
    o = np.asarray(o_dir, np.float64)
    o = (o / np.linalg.norm(o)).astype(np.float32)
    for a, ax in enumerate("xyz"):
        V["o" + ax] = np.full(n, o[a], np.float32)
    V["g"] = np.full(n, g, np.float32)
    V["e_delta"] = np.zeros(n, np.uint8)
    return V


def _in_degree(nbr):
    valid = nbr >= 0
    return np.bincount(nbr[valid], minlength=nbr.shape[0]).astype(np.float64)


@pytest.mark.parametrize("g", [0.0, 0.7])
def test_direct_weights_identical_lobes_closed_form_on_knn_graphs(g):
    """Eq. ag-direct on a kNN graph whose |R(j)| vary, continuous emitter
    (pe_e > 0) and phase samples (pe_ph > 0): with one lobe rho for every
    vertex the marginals are K_j rho, so
      Ae_{s,j}  = sigma_s rho(e_j) / (K_j (rho(e_j) + pe_e_j)),
      Aph_{s,j} = sigma_s rho(d_j) / (K_j (rho(d_j) + pe_ph_j)),
      A+_{s,j}  = sigma_s / K_j,
    with K_j = |R(j)|; for g = 0 this is sigma_s / (4 pi) / (K_j / (4 pi) + K_j pe)."""
    n, k = 900, 8
    V = _identical_lobe_records(n, 31, g)
    rng = np.random.default_rng(32)
    V["pe_e"] = rng.uniform(0.01, 0.6, n).astype(np.float32)
    V["pe_ph"] = rng.uniform(0.01, 0.6, n).astype(np.float32)
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, k)
    agg = oracle.aggregate(V, nbr)
    Kj = _in_degree(nbr)[nbr]
    Ns = (nbr >= 0).sum(axis=1)[:, None].astype(np.float64)
    assert (Kj != Ns).mean() > 0.5  # the two counts differ on most entries
    X = oracle.vertex_arrays(V)
    sig = X["sigma_s"][:, None]
    o = X["o"][0]
    if g == 0.0:
        pe, pph = X["pe_e"][nbr], X["pe_ph"][nbr]
        np.testing.assert_allclose(agg["Ae"], sig / FOUR_PI / (Kj / FOUR_PI + Kj * pe), rtol=1e-13)
        np.testing.assert_allclose(agg["Aph"], sig / FOUR_PI / (Kj / FOUR_PI + Kj * pph), rtol=1e-13)
    # the lobe from the pinned HG evaluation, at the sample directions only
    rho_e = oracle.hg(o, X["e"][nbr], X["g"][0])
    rho_d = oracle.hg(o, X["d"][nbr], X["g"][0])
    np.testing.assert_allclose(agg["Ae"], sig * rho_e / (Kj * (rho_e + X["pe_e"][nbr])), rtol=1e-12)
    np.testing.assert_allclose(agg["Aph"], sig * rho_d / (Kj * (rho_d + X["pe_ph"][nbr])), rtol=1e-12)
    np.testing.assert_allclose(agg["A"], sig / Kj, rtol=1e-12)


def _environment_records(n, seed, g, a_env, b_pdf):
    """Identical-lobe records on a kNN graph lit by an environment
    L(w) = 1 + a.w, with emitter samples drawn from pe(w) = (1 + b.w)/(4 pi)
    (rejection from the uniform sphere) and phase samples from the lobe."""
    V = _identical_lobe_records(n, seed, g)
    rng = np.random.default_rng(seed + 1)
    V["sigma_s"] = np.ones(n, np.float32)
    o = np.stack([V["ox"], V["oy"], V["oz"]], axis=1).astype(np.float64)
    d = _hg_sample(rng, o, np.full(n, float(np.float32(g))))
    e = np.empty((n, 3))
    todo = np.arange(n)
    bmax = 1 + np.linalg.norm(b_pdf)
    while todo.size:
        w = synthetic.unit_vectors(rng, todo.size).astype(np.float64)
        acc = rng.uniform(size=todo.size) * bmax < 1 + w @ b_pdf
        e[todo[acc]] = w[acc]
        todo = todo[~acc]
    # directions are stored as float32; evaluate L and pe at the stored values
    d32, e32 = d.astype(np.float32), e.astype(np.float32)
    for a, ax in enumerate("xyz"):
        V["d" + ax] = np.ascontiguousarray(d32[:, a])
        V["e" + ax] = np.ascontiguousarray(e32[:, a])
    d64, e64 = d32.astype(np.float64), e32.astype(np.float64)
    V["Le"] = 1 + e64 @ a_env
    V["pe_e"] = (1 + e64 @ b_pdf) / FOUR_PI
    V["Lph"] = 1 + d64 @ a_env
    V["pe_ph"] = (1 + d64 @ b_pdf) / FOUR_PI
    return V


def test_direct_term_unbiased_over_receivers_on_knn_graphs():
    """Each sample j's emitter and phase samples, weighted over the receivers
    R(j) that use them, estimate integral(rho L) without bias when the lobes
    are identical: E[sum_{s in R(j)} (A°_{s,2j} Le_j + A°_{s,2j+1} Lph_j)]
    = sigma (1 - g a.o) for every j, whatever |R(j)|. Checked on the per-sample
    totals of a 100 000-vertex kNN graph (|z| < 5)."""
    n, k, g = 100_000, 8, 0.3
    a_env = np.array([0.3, -0.5, 0.4])
    b_pdf = np.array([-0.6, 0.2, 0.5])
    V = _environment_records(n, 51, g, a_env, b_pdf)
    q = oracle.quantize(V["px"], V["py"], V["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, k)
    indeg = _in_degree(nbr)
    assert indeg.std() > 1.0  # receivers per sample vary widely
    agg = oracle.aggregate(V, nbr)
    X = oracle.vertex_arrays(V)
    valid = nbr >= 0
    j = np.where(valid, nbr, 0)
    contrib = agg["Ae"] * X["Le"][j] + agg["Aph"] * X["Lph"][j]
    t = np.bincount(nbr[valid], weights=contrib[valid], minlength=n)
    o = X["o"][0]
    expect = float(np.float32(g)) * -1.0 * (o @ a_env) + 1.0
    z = (t - expect).mean() / ((t - expect).std() / np.sqrt(n))
    assert abs(z) < 5, z
