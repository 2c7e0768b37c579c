"""Seeded synthetic vertex sets with a prescribed structure.

Input generators for tests (no path-graph arithmetic): clustered point sets
whose k-nearest-neighbour sets are exactly the clusters, cyclic successor
chains (an "infinite medium" with no path ends), random unit directions and
light records. All arrays are float32 / int32 / uint8 like the recorder's.
"""
from __future__ import annotations

import numpy as np


def unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


def clustered_vertices(n_clusters: int, k: int, seed: int = 0, *, g=0.0, albedo=0.9, sigma_t=3.0,
                       spread=1e-3, spacing=0.1, cyclic=True, delta=False, Le=1.0, pe_e=0.0,
                       Lph=0.0, pe_ph=0.0, random_g=False, random_sigma=False, L0=0.0) -> dict:
    """n_clusters groups of exactly k points.

    Group centres sit on a lattice with ``spacing``; members lie within
    ``spread`` of their centre, so each point's k nearest neighbours (itself
    included) are its own group. ``cyclic`` links every vertex to a successor
    so no path ends (succ is a random permutation cycle).
    """
    rng = np.random.default_rng(seed)
    n = n_clusters * k
    side = int(np.ceil(n_clusters ** (1 / 3)))
    cid = np.repeat(np.arange(n_clusters), k)
    cx, cy, cz = cid % side, (cid // side) % side, cid // (side * side)
    centre = 0.05 + spacing * np.stack([cx, cy, cz], axis=1)
    pos = centre + spread * rng.uniform(-1, 1, size=(n, 3))
    V = dict(px=pos[:, 0].astype(np.float32), py=pos[:, 1].astype(np.float32), pz=pos[:, 2].astype(np.float32))
    o, d, e = unit_vectors(rng, n), unit_vectors(rng, n), unit_vectors(rng, n)
    for name, arr in (("o", o), ("d", d), ("e", e)):
        for a, ax in enumerate("xyz"):
            V[name + ax] = np.ascontiguousarray(arr[:, a])
    V["g"] = (rng.uniform(-0.5, 0.9, n) if random_g else np.full(n, g)).astype(np.float32)
    st = rng.uniform(1.0, 5.0, n) if random_sigma else np.full(n, sigma_t)
    V["sigma_t"] = st.astype(np.float32)
    V["sigma_s"] = (albedo * V["sigma_t"].astype(np.float64)).astype(np.float32)
    V["w_prop"] = (1.0 / V["sigma_t"].astype(np.float64)).astype(np.float32)
    V["Le"] = np.full(n, Le, np.float32)
    V["pe_e"] = np.full(n, pe_e, np.float32)
    V["Lph"] = np.full(n, Lph, np.float32)
    V["pe_ph"] = np.full(n, pe_ph, np.float32)
    V["e_delta"] = np.full(n, 1 if delta else 0, np.uint8)
    if cyclic:
        perm = rng.permutation(n)
        succ = np.empty(n, np.int32)
        succ[perm] = np.roll(perm, -1)
    else:
        succ = -np.ones(n, np.int32)
    V["succ"] = succ
    V["L0"] = np.full(n, L0, np.float32)
    V["voxel"] = np.zeros(n, np.int32)
    V["n"] = n
    V["cluster"] = cid
    return V


def random_records(n: int, seed: int = 0, *, n_paths: int | None = None, max_len: int = 6) -> dict:
    """Random vertex records grouped into paths of random length (1..max_len).

    Directions, coefficients and light records are random; about half of the
    emitter samples are delta lights. Returns the per-vertex arrays plus
    per-path ``first``/``bg``.
    """
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(n, 3))
    V = dict(px=pos[:, 0].astype(np.float32), py=pos[:, 1].astype(np.float32), pz=pos[:, 2].astype(np.float32))
    o, d, e = unit_vectors(rng, n), unit_vectors(rng, n), unit_vectors(rng, n)
    for name, arr in (("o", o), ("d", d), ("e", e)):
        for a, ax in enumerate("xyz"):
            V[name + ax] = np.ascontiguousarray(arr[:, a])
    V["g"] = rng.uniform(-0.3, 0.9, n).astype(np.float32)
    V["sigma_t"] = rng.uniform(1.0, 10.0, n).astype(np.float32)
    V["sigma_s"] = (rng.uniform(0.5, 0.99, n) * V["sigma_t"]).astype(np.float32)
    V["w_prop"] = (1.0 / V["sigma_t"].astype(np.float64)).astype(np.float32)
    V["e_delta"] = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    V["Le"] = rng.uniform(0.0, 2.0, n).astype(np.float32)
    V["pe_e"] = np.where(V["e_delta"] == 1, 0.0, rng.uniform(0.01, 1.0, n)).astype(np.float32)
    hit = rng.uniform(size=n) < 0.3
    V["Lph"] = np.where(hit, rng.uniform(0.0, 1.0, n), 0.0).astype(np.float32)
    V["pe_ph"] = np.where(hit, rng.uniform(0.01, 1.0, n), 0.0).astype(np.float32)
    V["L0"] = rng.uniform(0.0, 1.0, n).astype(np.float32)
    V["voxel"] = rng.integers(0, 64, n).astype(np.int32)
    # paths: consecutive runs
    succ = -np.ones(n, np.int32)
    firsts = []
    v = 0
    while v < n:
        ln = int(rng.integers(1, max_len + 1))
        ln = min(ln, n - v)
        firsts.append(v)
        for u in range(v, v + ln - 1):
            succ[u] = u + 1
        v += ln
    V["succ"] = succ
    V["n"] = n
    if n_paths is None:
        n_paths = len(firsts)
    first = -np.ones(n_paths, np.int32)
    m = min(n_paths, len(firsts))
    # scatter the paths over path slots; some slots stay empty (escaped camera rays)
    slots = np.sort(rng.choice(n_paths, size=m, replace=False)) if n_paths > m else np.arange(m)
    first[slots] = np.array(firsts[:m], np.int32)
    V["first"] = first
    V["bg"] = np.where(first < 0, rng.uniform(0.0, 1.0, n_paths), 0.0).astype(np.float32)
    return V


def random_extra(n_paths: int, M: int, seed: int = 0) -> dict:
    """Random extra first-vertex emitter samples, M per path (the recorder's
    x_* arrays): random directions, about half of them delta lights."""
    rng = np.random.default_rng(seed)
    q = n_paths * M
    e = unit_vectors(rng, q)
    delta = (rng.uniform(size=q) < 0.5).astype(np.uint8)
    return {"x_ex": np.ascontiguousarray(e[:, 0]), "x_ey": np.ascontiguousarray(e[:, 1]),
            "x_ez": np.ascontiguousarray(e[:, 2]), "x_Le": rng.uniform(0.0, 2.0, q).astype(np.float32),
            "x_pe": np.where(delta == 1, 0.0, rng.uniform(0.01, 1.0, q)).astype(np.float32),
            "x_delta": delta, "extra_direct": M}
