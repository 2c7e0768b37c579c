#!/usr/bin/env python3
"""Writes tests/golden/cloud128_oracle_image.txt: the FP64 oracle's image of the
heterogeneous-cloud workload at full size (128^3 fBm medium, albedo 0.99,
HG g = 0.8, sun + sky, 256 x 256 pixels, 16 spp, depth 64, 8.7 M vertices;
k = 16, 30 sweeps): the central 64 x 64 crop, every 8th pixel in x and y of
the whole image, and the 30 sweep residuals, with a checksum of the traced
inputs so a reader can tell the file belongs to the recorder's output.

Only oracle/ computes: the seeded recorder supplies the inputs; the sample
marginals are formed once (oracle.sample_marginals) and the aggregation rows
are split over spawned worker processes, each calling oracle.aggregate on its
rows with those marginals (the same arithmetic as one call over all rows).

  python tests/golden/make_cloud128_reference.py [--workers N]
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(ROOT, "tests", "golden", "cloud128_oracle_image.txt")
CROP = (96, 96, 64)  # y0, x0, size
STRIDE = 8


def trace_checksum(rec) -> str:
    h = hashlib.sha256()
    for k in sorted(rec):
        v = rec[k]
        if isinstance(v, np.ndarray):
            h.update(k.encode())
            h.update(np.ascontiguousarray(v).tobytes())
    return h.hexdigest()


def _agg_rows(args):
    path, a, b = args
    import oracle

    z = np.load(path, mmap_mode="r")
    skip = ("nbr", "pm_d", "pm_e", "Kj")
    V = {k: np.asarray(z[k]) for k in z.files if k not in skip}
    marg = (np.asarray(z["pm_d"]), np.asarray(z["pm_e"]), np.asarray(z["Kj"]))
    out = oracle.aggregate(V, np.asarray(z["nbr"]), rows=np.arange(a, b), marginals=marg)
    return a, b, out["A"], out["c"], out["D"]


def main():
    import oracle
    import pgrec

    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    t0 = time.time()
    sc = pgrec.CLOUD128
    rec = pgrec.trace(sc)
    n = rec["n"]
    digest = trace_checksum(rec)
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, sc.k, workers=args.workers)
    print(f"traced {n} vertices, kNN done ({time.time() - t0:.0f} s)", flush=True)
    A = np.zeros((n, sc.k))
    c = np.zeros(n)
    D = np.zeros(n)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "inputs.npz")
        fields = {k: v for k, v in rec.items() if isinstance(v, np.ndarray) and len(v) == n}
        pm_d, pm_e, Kj = oracle.sample_marginals(rec, nbr)
        print(f"marginals ({time.time() - t0:.0f} s)", flush=True)
        np.savez(path, nbr=nbr, pm_d=pm_d, pm_e=pm_e, Kj=Kj, **fields)
        step = 65536
        jobs = [(path, a, min(n, a + step)) for a in range(0, n, step)]
        with mp.get_context("spawn").Pool(args.workers) as pool:
            for a, b, Aa, ca, Da in pool.imap_unordered(_agg_rows, jobs):
                A[a:b], c[a:b], D[a:b] = Aa, ca, Da
    print(f"aggregated ({time.time() - t0:.0f} s)", flush=True)
    L, _, res = oracle.propagate(rec, nbr, A, c, rec["L0"], sc.iters)
    img = oracle.gather(rec, nbr, A, L, D, rec["first"], rec["bg"], sc.spp, sc.width, sc.height)
    print(f"propagated and gathered ({time.time() - t0:.0f} s)", flush=True)
    y0, x0, s = CROP
    with open(OUT, "w") as f:
        f.write(f"# FP64 oracle image of {sc.name} ({sc.width}x{sc.height}, {sc.spp} spp, k={sc.k}, "
                f"{sc.iters} sweeps, {n} vertices)\n")
        f.write("# written by tests/golden/make_cloud128_reference.py (oracle/ only; inputs from the seeded recorder)\n")
        f.write(f"trace_sha256 {digest}\n")
        f.write("residuals " + " ".join(f"{r:.17g}" for r in res) + "\n")
        f.write(f"crop {y0} {x0} {s}\n")
        for yy in range(y0, y0 + s):
            f.write(" ".join(f"{v:.17g}" for v in img[yy, x0:x0 + s]) + "\n")
        f.write(f"stride {STRIDE}\n")
        for yy in range(0, sc.height, STRIDE):
            f.write(" ".join(f"{v:.17g}" for v in img[yy, ::STRIDE]) + "\n")
    print(f"wrote {OUT} ({time.time() - t0:.0f} s)")


def load():
    """Parsed file: dict(trace_sha256, residuals, crop=(y0, x0, array), stride=(s, array))."""
    with open(OUT) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    out = {"trace_sha256": lines[0].split()[1],
           "residuals": np.array([float(v) for v in lines[1].split()[1:]])}
    _, y0, x0, s = lines[2].split()
    y0, x0, s = int(y0), int(x0), int(s)
    crop = np.array([[float(v) for v in ln.split()] for ln in lines[3:3 + s]])
    st = int(lines[3 + s].split()[1])
    strided = np.array([[float(v) for v in ln.split()] for ln in lines[4 + s:]])
    out["crop"] = (y0, x0, crop)
    out["stride"] = (st, strided)
    return out


if __name__ == "__main__":
    main()
