#!/usr/bin/env python3
"""Writes tests/golden/dense256_oracle_image.txt: the FP64 oracle's image of
the large dense workload at full size (256^3 fBm medium, sigma_t up to 60,
albedo 0.999, HG g = 0.9, rectangular area light + constant environment,
1024 x 1024 pixels, 8 spp, depth 256, 158.7 M vertices; k = 16, 50 sweeps)
at sampled pixels: the central 64 x 64 crop and every 32nd pixel in x and y,
with a checksum of the traced inputs.

The whole graph has to be solved (every sweep couples all vertices), and its
FP64 arrays (2.5e9 neighbour entries) do not fit in memory, so the work is
streamed in row blocks through disk-backed arrays, and only oracle/ computes:
  * kNN: oracle.knn over row blocks, with one k-d tree built once;
  * the sample marginals: oracle.sample_marginals on each row block's
    sub-problem (the block's receivers and the samples they use, re-indexed),
    the blocks' partial sums added (a reordering of the same float64 sums);
  * the weights: oracle.aggregate(rows=...) on the same sub-problems with
    the global marginals;
  * each sweep: oracle.sweep on each row block with every receiver as its own
    successor (so it returns w_s (A+ L+ + c)_s of the block's receivers),
    then oracle.sweep over the identity table to move those values to the
    predecessors (a product with 1.0 and a sum with 0.0, both exact);
  * the sampled pixels: oracle.gather on the sampled paths' first vertices.
The blocks run in spawned worker processes.

  python tests/golden/make_dense256_reference.py [--workers N] [--workdir DIR]
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import shutil
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(ROOT, "tests", "golden", "dense256_oracle_image.txt")
CROP = (480, 480, 64)  # y0, x0, size
STRIDE = 32
BLOCK = 500_000
# vertex fields the oracle's aggregation reads
AGG_FIELDS = ("ox", "oy", "oz", "dx", "dy", "dz", "ex", "ey", "ez", "g", "sigma_s", "sigma_t", "w_prop", "Le",
              "pe_e", "Lph", "pe_ph", "e_delta", "succ")
CHECK_FIELDS = ("px", "py", "pz", "succ", "L0", "first", "bg")


def trace_checksum(rec) -> str:
    """sha256 over the positions, successors, L0, first vertices and
    backgrounds (enough to tell that a trace is this one)."""
    h = hashlib.sha256()
    for k in CHECK_FIELDS:
        a = np.asarray(rec[k])
        h.update(k.encode())
        for i in range(0, len(a), 1 << 24):
            h.update(np.ascontiguousarray(a[i:i + (1 << 24)]).tobytes())
    return h.hexdigest()


def sample_pixels(width, height):
    """Pixel indices (y * width + x) of the central crop, then the strided grid."""
    y0, x0, s = CROP
    crop = (np.arange(y0, y0 + s)[:, None] * width + np.arange(x0, x0 + s)[None, :]).reshape(-1)
    grid = (np.arange(0, height, STRIDE)[:, None] * width + np.arange(0, width, STRIDE)[None, :]).reshape(-1)
    return crop, grid


class Store:
    """Disk-backed arrays (.npy memmaps) in one directory."""

    def __init__(self, d):
        self.d = d

    def path(self, name):
        return os.path.join(self.d, name + ".npy")

    def new(self, name, shape, dtype):
        return np.lib.format.open_memmap(self.path(name), mode="w+", dtype=dtype, shape=shape)

    def get(self, name, mode="r"):
        return np.load(self.path(name), mmap_mode=mode)


def _subproblem(st, a, b, fields):
    """Records of receivers a..b-1 and of the samples their rows use,
    re-indexed: local vertices 0..B-1 are the receivers, the table's entries
    point at local indices. Returns (verts, V_sub, nbr_local)."""
    nb = np.asarray(st.get("nbr")[a:b], np.int64)
    rows = np.arange(a, b)
    used = np.unique(nb[nb >= 0])
    extra = np.setdiff1d(used, rows, assume_unique=True)
    verts = np.concatenate([rows, extra])
    order = np.argsort(verts, kind="stable")
    sv = verts[order]
    loc = np.where(nb >= 0, order[np.searchsorted(sv, np.where(nb >= 0, nb, 0))], -1)
    V = {}
    for f in fields:
        arr = st.get(f)
        V[f] = np.asarray(arr[verts]) if f != "succ" else np.full(len(verts), -1, np.int32)
    return verts, V, loc


def _marginals_block(args):
    d, a, b = args
    import oracle

    st = Store(d)
    verts, V, loc = _subproblem(st, a, b, AGG_FIELDS)
    pm_d, pm_e, K = oracle.sample_marginals(V, loc)
    keep = K > 0
    return verts[keep], pm_d[keep], pm_e[keep], K[keep]


def _aggregate_block(args):
    d, a, b = args
    import oracle

    st = Store(d)
    verts, V, loc = _subproblem(st, a, b, AGG_FIELDS)
    marg = tuple(np.asarray(st.get(m)[verts]) for m in ("pm_d", "pm_e", "Kj"))
    out = oracle.aggregate(V, loc, rows=np.arange(b - a), marginals=marg)
    A = st.get("A", "r+")
    A[a:b] = out["A"]
    A.flush()
    c = st.get("c", "r+")
    c[a:b] = out["c"]
    c.flush()
    D = st.get("D", "r+")
    D[a:b] = out["D"]
    D.flush()
    return b - a


def _sweep_block(args):
    d, a, b, t = args
    import oracle

    st = Store(d)
    L = st.get(f"L{t % 2}")
    w = st.get("w_prop")
    # every receiver its own successor: oracle.sweep returns w_s (A+ L + c)_s
    V = {"succ": np.arange(b - a, dtype=np.int64), "w_prop": np.asarray(w[a:b])}
    y = oracle.sweep(V, np.asarray(st.get("nbr")[a:b], np.int64), np.asarray(st.get("A")[a:b]),
                     np.asarray(st.get("c")[a:b]), L)
    out = st.get("y", "r+")
    out[a:b] = y
    out.flush()
    return b - a


def _knn_block(args):
    d, a, b, k = args
    import oracle

    nb = oracle.knn(_KNN["q"], k, workers=1, rows=np.arange(a, b), tree=_KNN["tree"])
    out = Store(d).get("nbr", "r+")
    out[a:b] = nb.astype(np.int32)
    out.flush()
    return b - a


# the quantised points and their k-d tree, built once in the parent and
# shared with the forked kNN workers
_KNN = {}


def solve(sc, pix, workers, workdir=None, log=print):
    """The oracle's image of scene ``sc`` at pixel indices ``pix`` (y * width
    + x), streamed as described above. Returns (n, trace digest, values)."""
    import oracle
    import pgrec
    from scipy.spatial import cKDTree

    d = tempfile.mkdtemp(prefix="dense256_", dir=workdir)
    st = Store(d)
    ctx = mp.get_context("spawn")
    try:
        names = iter(range(1 << 30))
        rec = pgrec.trace(sc, alloc=lambda shape, dtype: st.new(f"tr{next(names)}", shape, dtype))
        n, k, T = rec["n"], sc.k, sc.iters
        for f in AGG_FIELDS + ("px", "py", "pz", "L0"):
            os.link(rec[f].filename, st.path(f))
        digest = trace_checksum(rec)
        log(f"traced {n} vertices")
        _KNN["q"] = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
        _KNN["tree"] = cKDTree(_KNN["q"].astype(np.float64))
        log("k-d tree")
        st.new("nbr", (n, k), np.int32).flush()
        blocks = [(a, min(n, a + BLOCK)) for a in range(0, n, BLOCK)]
        with mp.get_context("fork").Pool(workers) as pool:
            for _ in pool.imap_unordered(_knn_block, [(d, a, b, k) for a, b in blocks]):
                pass
        _KNN.clear()
        log("kNN")
        pm = {m: np.zeros(n) for m in ("pm_d", "pm_e", "Kj")}
        with ctx.Pool(workers) as pool:
            for verts, p1, p2, p3 in pool.imap_unordered(_marginals_block, [(d, a, b) for a, b in blocks]):
                pm["pm_d"][verts] += p1
                pm["pm_e"][verts] += p2
                pm["Kj"][verts] += p3
        for m, v in pm.items():
            np.save(st.path(m), v)
        del pm
        log("sample marginals")
        st.new("A", (n, k), np.float64).flush()
        st.new("c", (n,), np.float64).flush()
        st.new("D", (n,), np.float64).flush()
        with ctx.Pool(workers) as pool:
            for _ in pool.imap_unordered(_aggregate_block, [(d, a, b) for a, b in blocks]):
                pass
        log("aggregation")
        succ = np.asarray(rec["succ"], np.int64)
        # L+ at sweep 0 (path ends set to zero), from oracle.propagate with no sweep
        L, _, _ = oracle.propagate({"succ": succ}, None, None, None, rec["L0"], 0)
        ident = np.arange(n, dtype=np.int64)[:, None]
        ones = np.ones((n, 1))
        zeros = np.zeros(n)
        vmap = {"succ": succ, "w_prop": np.ones(n)}
        st.new("y", (n,), np.float64).flush()
        with ctx.Pool(workers) as pool:
            for t in range(T):
                np.save(st.path(f"L{t % 2}"), L)
                for _ in pool.imap_unordered(_sweep_block, [(d, a, b, t) for a, b in blocks]):
                    pass
                # y of each receiver to its predecessor (exact: 1.0 * y + 0.0)
                L = oracle.sweep(vmap, ident, ones, zeros, np.asarray(st.get("y")))
                log(f"sweep {t + 1}")
        del ident, ones, zeros, vmap
        paths = (np.asarray(pix)[:, None] * sc.spp + np.arange(sc.spp)[None, :]).reshape(-1)
        first = np.asarray(rec["first"])[paths].astype(np.int64)
        F = np.unique(first[first >= 0])
        first_loc = np.where(first >= 0, np.searchsorted(F, np.where(first >= 0, first, 0)), -1)
        VF = {"w_prop": np.asarray(st.get("w_prop")[F])}
        img = oracle.gather(VF, np.asarray(st.get("nbr")[F], np.int64), np.asarray(st.get("A")[F]), L,
                            np.asarray(st.get("D")[F]), first_loc, np.asarray(rec["bg"])[paths], sc.spp, len(pix), 1)
        log("sampled pixels")
        return n, digest, img.reshape(-1)
    finally:
        shutil.rmtree(d, ignore_errors=True)


def main():
    import pgrec

    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--workdir", default=None, help="directory for the disk-backed arrays (about 60 GB)")
    args = ap.parse_args()
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.0f} s] {m}", flush=True)  # noqa: E731
    sc = pgrec.CLOUD256_DENSE
    crop, grid = sample_pixels(sc.width, sc.height)
    n, digest, img = solve(sc, np.concatenate([crop, grid]), args.workers, args.workdir, log)
    y0, x0, s = CROP
    with open(OUT, "w") as f:
        f.write(f"# FP64 oracle image of {sc.name} ({sc.width}x{sc.height}, {sc.spp} spp, k={sc.k}, "
                f"{sc.iters} sweeps, {n} vertices) at sampled pixels\n")
        f.write("# written by tests/golden/make_dense256_reference.py (oracle/ only; inputs from the seeded "
                "recorder)\n")
        f.write(f"trace_sha256 {digest}\n")
        f.write(f"crop {y0} {x0} {s}\n")
        for r in range(s):
            f.write(" ".join(f"{v:.17g}" for v in img[r * s:(r + 1) * s]) + "\n")
        m = sc.width // STRIDE
        f.write(f"stride {STRIDE}\n")
        g = img[s * s:]
        for r in range(sc.height // STRIDE):
            f.write(" ".join(f"{v:.17g}" for v in g[r * m:(r + 1) * m]) + "\n")
    log(f"wrote {OUT}")


def load():
    """Parsed file: dict(trace_sha256, crop=(y0, x0, array), stride=(s, array))."""
    with open(OUT) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    out = {"trace_sha256": lines[0].split()[1]}
    _, y0, x0, s = lines[1].split()
    y0, x0, s = int(y0), int(x0), int(s)
    out["crop"] = (y0, x0, np.array([[float(v) for v in ln.split()] for ln in lines[2:2 + s]]))
    st = int(lines[2 + s].split()[1])
    out["stride"] = (st, np.array([[float(v) for v in ln.split()] for ln in lines[3 + s:]]))
    return out


if __name__ == "__main__":
    main()
