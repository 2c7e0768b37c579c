#!/usr/bin/env python3
"""Writes tests/golden/cloud64_oracle_grad.txt: the FP64 oracle's per-voxel
albedo gradient of the differentiation workload at full size (64^3 fBm
medium, albedo 0.95, HG g = 0.6, sun + sky, 128 x 128 pixels, 8 spp, depth
32, about 1.03 M vertices; k = 16, 20 sweeps).

The loss is L = 1/2 sum_p (I_p - I*_p)^2 against a seeded target render: the
same pipeline with the per-voxel albedo perturbed by u_x, u_x uniform in
[-0.03, 0.03] (numpy default_rng(TARGET_SEED), one draw per voxel). On 64
occupied voxels (numpy default_rng(VOXEL_SEED), drawn without replacement
from the sorted occupied voxels) the file holds, per voxel:
  * the central difference (L(a + h e_x) - L(a - h e_x)) / (2 h), h = 1e-3,
    each voxel perturbed on its own (sigma_s = albedo * sigma_t of that
    voxel's vertices moves by +-h sigma_t), the graph, paths and L0 fixed;
  * the oracle's adjoint (oracle.adjoint) at the same voxels.
Also the loss, the oracle's image and the target at every 4th pixel in x
and y, the 20 sweep residuals, and a checksum of the traced inputs.

Only oracle/ computes: the seeded recorder supplies the inputs; the sample
marginals are formed once (oracle.sample_marginals: they do not depend on
sigma_s); a perturbed voxel's rows are re-aggregated with oracle.aggregate
(rows=...) and every difference runs oracle.propagate and oracle.gather in
full. The differences are split over spawned worker processes.

  python tests/golden/make_cloud64_reference.py [--workers N]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

OUT = os.path.join(ROOT, "tests", "golden", "cloud64_oracle_grad.txt")
TARGET_SEED = 2024
VOXEL_SEED = 11894
N_VOXELS = 64
H = 1e-3
STRIDE = 4


def target_albedo_offsets(grid_res):
    """The target render's per-voxel albedo offsets (input generator)."""
    return np.random.default_rng(TARGET_SEED).uniform(-0.03, 0.03, grid_res ** 3)


def pick_voxels(voxel):
    """The 64 checked voxels: a seeded draw among the occupied ones."""
    occ = np.unique(np.asarray(voxel, np.int64))
    return np.random.default_rng(VOXEL_SEED).choice(occ, N_VOXELS, replace=False)


def _load(path):
    z = np.load(path, mmap_mode="r")
    skip = ("nbr", "pm_d", "pm_e", "Kj", "A", "c", "D", "target", "first", "bg")
    V = {k: np.asarray(z[k]) for k in z.files if k not in skip}
    return z, V


def _fd_voxels(args):
    path, voxels, spp, width, height, iters = args
    import oracle

    z, V = _load(path)
    nbr = np.asarray(z["nbr"])
    marg = (np.asarray(z["pm_d"]), np.asarray(z["pm_e"]), np.asarray(z["Kj"]))
    A0, c0, D0 = np.asarray(z["A"]), np.asarray(z["c"]), np.asarray(z["D"])
    first, bg, target = np.asarray(z["first"]), np.asarray(z["bg"]), np.asarray(z["target"])
    sig0 = np.asarray(V["sigma_s"], np.float64)
    st = np.asarray(V["sigma_t"], np.float64)
    vox = np.asarray(V["voxel"], np.int64)
    out = []
    for x in voxels:
        rows = np.nonzero(vox == x)[0]
        losses = []
        for sgn in (1.0, -1.0):
            sig = sig0.copy()
            sig[rows] += sgn * H * st[rows]
            part = oracle.aggregate(V, nbr, sigma_s=sig, rows=rows, marginals=marg)
            A, c, D = A0.copy(), c0.copy(), D0.copy()
            A[rows], c[rows], D[rows] = part["A"], part["c"], part["D"]
            L, _, _ = oracle.propagate(V, nbr, A, c, V["L0"], iters)
            img = oracle.gather(V, nbr, A, L, D, first, bg, spp, width, height)
            losses.append(oracle.image_loss(img, target)[0])
        out.append((int(x), (losses[0] - losses[1]) / (2 * H)))
    return out


def _agg_rows(args):
    path, a, b, which = args
    import oracle

    z, V = _load(path)
    sig = np.asarray(z["sigma_tgt"]) if which == "target" else None
    marg = (np.asarray(z["pm_d"]), np.asarray(z["pm_e"]), np.asarray(z["Kj"]))
    out = oracle.aggregate(V, np.asarray(z["nbr"]), sigma_s=sig, rows=np.arange(a, b), marginals=marg)
    return a, b, out["A"], out["c"], out["D"]


def _aggregate_all(pool, path, n, k, which):
    A = np.zeros((n, k))
    c = np.zeros(n)
    D = np.zeros(n)
    step = 32768
    jobs = [(path, a, min(n, a + step), which) for a in range(0, n, step)]
    for a, b, Aa, ca, Da in pool.imap_unordered(_agg_rows, jobs):
        A[a:b], c[a:b], D[a:b] = Aa, ca, Da
    return A, c, D


def main():
    import oracle
    import pgrec
    from make_cloud128_reference import trace_checksum

    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    t0 = time.time()
    sc = pgrec.CLOUD64_GRAD
    rec = pgrec.trace(sc)
    n = rec["n"]
    digest = trace_checksum(rec)
    q = oracle.quantize(rec["px"], rec["py"], rec["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, sc.k, workers=args.workers)
    pm_d, pm_e, Kj = oracle.sample_marginals(rec, nbr)
    print(f"traced {n} vertices, kNN and marginals ({time.time() - t0:.0f} s)", flush=True)
    st = rec["sigma_t"].astype(np.float64)
    sig_tgt = (sc.albedo + target_albedo_offsets(sc.grid_res)[rec["voxel"]]) * st
    fields = {k: v for k, v in rec.items() if isinstance(v, np.ndarray) and len(v) == n}
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as td, ctx.Pool(args.workers) as pool:
        path = os.path.join(td, "inputs.npz")
        np.savez(path, nbr=nbr, pm_d=pm_d, pm_e=pm_e, Kj=Kj, sigma_tgt=sig_tgt, **fields)
        At, ct, Dt = _aggregate_all(pool, path, n, sc.k, "target")
        Lt, _, _ = oracle.propagate(rec, nbr, At, ct, rec["L0"], sc.iters)
        target = oracle.gather(rec, nbr, At, Lt, Dt, rec["first"], rec["bg"], sc.spp, sc.width, sc.height)
        del At, ct, Dt, Lt
        A, c, D = _aggregate_all(pool, path, n, sc.k, "base")
        L, _, res = oracle.propagate(rec, nbr, A, c, rec["L0"], sc.iters)
        img = oracle.gather(rec, nbr, A, L, D, rec["first"], rec["bg"], sc.spp, sc.width, sc.height)
        loss, dI = oracle.image_loss(img, target)
        print(f"target and base renders, loss {loss:.6g} ({time.time() - t0:.0f} s)", flush=True)
        adj = oracle.adjoint(rec, nbr, sc.iters, rec["L0"], dI, rec["first"], rec["bg"], sc.spp, sc.width,
                             sc.height, voxel=rec["voxel"], n_vox=sc.grid_res ** 3)
        print(f"adjoint ({time.time() - t0:.0f} s)", flush=True)
        vox = pick_voxels(rec["voxel"])
        path2 = os.path.join(td, "fd.npz")
        np.savez(path2, nbr=nbr, pm_d=pm_d, pm_e=pm_e, Kj=Kj, A=A, c=c, D=D, target=target,
                 first=rec["first"], bg=rec["bg"], **fields)
        jobs = [(path2, vox[i::args.workers], sc.spp, sc.width, sc.height, sc.iters) for i in range(args.workers)]
        fd = {}
        for part in pool.imap_unordered(_fd_voxels, jobs):
            fd.update(dict(part))
    print(f"central differences ({time.time() - t0:.0f} s)", flush=True)
    with open(OUT, "w") as f:
        f.write(f"# FP64 oracle per-voxel albedo gradient of {sc.name} ({sc.width}x{sc.height}, {sc.spp} spp, "
                f"k={sc.k}, {sc.iters} sweeps, {n} vertices)\n")
        f.write("# written by tests/golden/make_cloud64_reference.py (oracle/ only; inputs from the seeded recorder)\n")
        f.write(f"trace_sha256 {digest}\n")
        f.write(f"target_seed {TARGET_SEED} voxel_seed {VOXEL_SEED} h {H!r}\n")
        f.write(f"loss {loss:.17g}\n")
        f.write("residuals " + " ".join(f"{r:.17g}" for r in res) + "\n")
        f.write("# voxel central_difference oracle_adjoint\n")
        for x in vox:
            f.write(f"{int(x)} {fd[int(x)]:.17g} {adj['grad_albedo'][x]:.17g}\n")
        f.write(f"stride {STRIDE}\n")
        for name, im in (("image", img), ("target", target)):
            f.write(name + "\n")
            for yy in range(0, sc.height, STRIDE):
                f.write(" ".join(f"{v:.17g}" for v in im[yy, ::STRIDE]) + "\n")
    print(f"wrote {OUT} ({time.time() - t0:.0f} s)")


def load():
    """Parsed file: dict(trace_sha256, loss, residuals, voxels, fd, adjoint,
    stride, image, target)."""
    with open(OUT) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    out = {"trace_sha256": lines[0].split()[1], "loss": float(lines[2].split()[1]),
           "residuals": np.array([float(v) for v in lines[3].split()[1:]])}
    rows = np.array([[float(v) for v in ln.split()] for ln in lines[4:4 + N_VOXELS]])
    out["voxels"] = rows[:, 0].astype(np.int64)
    out["fd"] = rows[:, 1]
    out["adjoint"] = rows[:, 2]
    i = 4 + N_VOXELS
    out["stride"] = int(lines[i].split()[1])
    m = 128 // out["stride"]
    out["image"] = np.array([[float(v) for v in ln.split()] for ln in lines[i + 2:i + 2 + m]])
    out["target"] = np.array([[float(v) for v in ln.split()] for ln in lines[i + 3 + m:i + 3 + 2 * m]])
    return out


if __name__ == "__main__":
    main()
