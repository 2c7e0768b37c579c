"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each mutation replaces one oracle function for the duration of a test with a
copy that has one deliberate error; the pin that should catch it must then
raise. This shows the pins constrain the oracle, not just re-run it.
"""
import numpy as np
import pytest

import oracle
import oracle.pathgraph as opg
import pgrec

from test_oracle_pins import (SMALL_SCENES, _cluster_graph, test_hg_forward_convention,
                              test_mis_weights_sum_to_one_on_knn_graphs)


def _k1_image(scene):
    rec = pgrec.trace(scene, nthreads=2)
    n = rec["n"]
    nbr = np.arange(n, dtype=np.int64)[:, None]
    agg = opg.aggregate(rec, nbr)
    L, _, _ = opg.propagate(rec, nbr, agg["A"], agg["c"], np.zeros(n), scene.max_depth)
    img = opg.gather(rec, nbr, agg["A"], L, agg["D"], rec["first"], rec["bg"], scene.spp, scene.width, scene.height)
    return img, rec["pt_image"]


def test_flipped_scattering_cosine_is_caught(monkeypatch):
    good = opg.hg

    def bad_hg(o, d, g):  # mu = +o.d instead of -o.d
        return good(o, -np.asarray(d, np.float64), g)

    monkeypatch.setattr(opg, "hg", bad_hg)
    monkeypatch.setattr(oracle, "hg", bad_hg)
    with pytest.raises(AssertionError):
        test_hg_forward_convention()
    img, pt = _k1_image(SMALL_SCENES[1])  # sun + sky: continuous-light MIS
    assert not np.allclose(img, pt, rtol=1e-12, atol=1e-15)


def test_wrong_propagation_weight_is_caught(monkeypatch):
    def bad_sweep(V, nbr, A, c, L):  # weight of the segment into v, not into succ(v)
        succ = np.asarray(V["succ"], np.int64)
        w = np.asarray(V["w_prop"], np.float64)
        Lj = np.where(nbr >= 0, L[np.where(nbr >= 0, nbr, 0)], 0.0)
        Lbar = (A * Lj).sum(axis=1) + c
        s = np.where(succ >= 0, succ, 0)
        return np.where(succ >= 0, w * Lbar[s], 0.0)

    monkeypatch.setattr(opg, "sweep", bad_sweep)
    img, pt = _k1_image(SMALL_SCENES[1])
    assert not np.allclose(img, pt, rtol=1e-12, atol=1e-15)


def test_transposed_numerator_is_caught():
    """Using the sample's own pdf rho_j(o_j, d_j) in the numerator instead of
    the receiver's rho_s(o_s, d_j) breaks the MIS identity of Eq. indirect-weight."""
    V, nbr = _cluster_graph(random_g=True, random_sigma=True, pe_e=0.0, pe_ph=0.0, Lph=1.0)
    X = opg.vertex_arrays(V)

    def col_sums(M):
        out = []
        for c in range(20):
            rows = np.nonzero(V["cluster"] == c)[0]
            col = {}
            for s in rows:
                for jj in range(nbr.shape[1]):
                    col[nbr[s, jj]] = col.get(nbr[s, jj], 0.0) + M[s, jj]
            out += list(col.values())
        return np.array(out)

    good = oracle.aggregate(V, nbr)["A"] / X["sigma_s"][:, None]
    np.testing.assert_allclose(col_sums(good), 1.0, rtol=1e-13)
    n, k = nbr.shape
    bad = np.zeros((n, k))
    for s in range(n):
        js = nbr[s]
        pm = opg.hg(X["o"][js][:, None, :], X["d"][js][None, :, :], X["g"][js][:, None]).sum(axis=0)
        bad[s] = opg.hg(X["o"][js], X["d"][js], X["g"][js]) / pm  # rho_j(o_j, d_j): wrong operand
    assert not np.allclose(col_sums(bad), 1.0, rtol=1e-6)


def test_receiver_neighbourhood_marginal_is_caught(monkeypatch):
    """Taking sample j's marginal over the receiver's own neighbourhood N(s)
    (the same thing on clusters) breaks the per-sample MIS sums on a kNN graph."""
    good = opg.aggregate

    def bad_aggregate(V, nbr, sigma_s=None, g=None, rows=None, marginals=None):
        out = good(V, nbr, sigma_s=sigma_s, g=g, rows=rows, marginals=marginals)
        X = opg.vertex_arrays(V)
        recv = np.arange(len(nbr)) if rows is None else np.asarray(rows)
        nb = nbr[recv]
        valid = nb >= 0
        j = np.where(valid, nb, 0)
        rho_ld = opg.hg(X["o"][j][:, :, None, :], X["d"][j][:, None, :, :], X["g"][j][:, :, None])
        pm = np.where(valid[:, :, None], rho_ld, 0.0).sum(axis=1)
        rho_sd = opg.hg(X["o"][recv][:, None, :], X["d"][j], X["g"][recv][:, None])
        out["A"] = np.where(valid, X["sigma_s"][recv][:, None] * rho_sd / pm, 0.0)
        return out

    monkeypatch.setattr(opg, "aggregate", bad_aggregate)
    monkeypatch.setattr(oracle, "aggregate", bad_aggregate)
    with pytest.raises(AssertionError):
        test_mis_weights_sum_to_one_on_knn_graphs()


def test_extra_direct_missing_sample_count_is_caught(monkeypatch):
    """Combining the M extra emitter samples as if each were alone (weight
    pe / (pe + rho) instead of M pe / (M pe + rho)) over-counts them."""
    from test_oracle_output_pins import test_extra_direct_expectation

    def bad_extra(V, first, X, M):
        X1 = {k: np.asarray(v) for k, v in X.items()}
        P = len(first)
        tot = np.zeros(P)
        for m in range(M):
            sub = {k: v.reshape(P, M)[:, m] for k, v in X1.items()}
            tot += good(V, first, sub, 1)
        return tot

    good = opg.extra_direct
    monkeypatch.setattr(oracle, "extra_direct", bad_extra)
    with pytest.raises(AssertionError):
        test_extra_direct_expectation(3)


def test_final_gather_marginal_without_receiver_is_caught(monkeypatch):
    """Leaving each sample's own strategy out of its marginal in the final
    gather biases the estimate."""
    from test_oracle_output_pins import test_final_gather_expectation

    good_hg = opg.hg
    calls = {"n": 0}

    def bad_hg(o, d, g):
        r = good_hg(o, d, g)
        calls["n"] += 1
        # the first phase evaluation of each chunk is the [p, l, j] marginal table
        if calls["n"] % 2 == 1 and np.ndim(r) == 3 and r.shape[1] == r.shape[2]:
            r = r.copy()
            idx = np.arange(r.shape[1])
            r[:, idx, idx] = 0.0
        return r

    monkeypatch.setattr(opg, "hg", bad_hg)
    with pytest.raises(AssertionError):
        test_final_gather_expectation()


def test_receiver_count_in_emitter_marginal_is_caught(monkeypatch):
    """Multiplying the emitter pdf inside the direct marginals of Eq. ag-direct
    by the receiver's |N(s)| instead of the sample's |R(j)| (the same count on
    clusters) fails the identical-lobe closed form and biases the Monte Carlo
    expectation of the direct term on a kNN graph."""
    from test_oracle_direct_pins import (test_direct_term_unbiased_over_receivers_on_knn_graphs,
                                         test_direct_weights_identical_lobes_closed_form_on_knn_graphs)

    good = opg.aggregate

    def bad_aggregate(V, nbr, sigma_s=None, g=None, rows=None, marginals=None):
        out = good(V, nbr, sigma_s=sigma_s, g=g, rows=rows, marginals=marginals)
        X = opg.vertex_arrays(V)
        if sigma_s is not None:
            X["sigma_s"] = np.asarray(sigma_s, np.float64)
        if g is not None:
            X["g"] = np.asarray(g, np.float64)
        recv = np.arange(len(nbr)) if rows is None else np.asarray(rows)
        nb = nbr[recv]
        valid = nb >= 0
        j = np.where(valid, nb, 0)
        Ks = valid.sum(axis=1).astype(np.float64)[:, None]
        sig, o, gs = X["sigma_s"][recv][:, None], X["o"][recv][:, None, :], X["g"][recv][:, None]
        rho_se = opg.hg(o, X["e"][j], gs)
        rho_sd = opg.hg(o, X["d"][j], gs)
        Ae = np.where(X["delta"][j], out["Ae"], sig * rho_se / (out["pm_e"][j] + Ks * X["pe_e"][j]))
        Aph = sig * rho_sd / (out["pm_d"][j] + Ks * X["pe_ph"][j])
        out["Ae"] = np.where(valid, Ae, 0.0)
        out["Aph"] = np.where(valid, Aph, 0.0)
        return out

    monkeypatch.setattr(opg, "aggregate", bad_aggregate)
    monkeypatch.setattr(oracle, "aggregate", bad_aggregate)
    for g in (0.0, 0.7):
        with pytest.raises(AssertionError):
            test_direct_weights_identical_lobes_closed_form_on_knn_graphs(g)
    with pytest.raises(AssertionError):
        test_direct_term_unbiased_over_receivers_on_knn_graphs()
