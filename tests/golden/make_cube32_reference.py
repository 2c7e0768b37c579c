#!/usr/bin/env python3
"""Writes tests/golden/cube32_oracle_image.txt: the FP64 oracle's image of the
plain-method workload (32^3 constant sigma_t = 2 in the unit cube, albedo
0.9, isotropic phase, one directional light, 64 x 64 pixels, 4 spp, depth 8,
delta tracking, seed 0; k = 8, 10 sweeps), every pixel, with the sweep
residuals and a checksum of the traced inputs.

Only oracle/ computes (oracle.forward on the seeded recorder's records).

  python tests/golden/make_cube32_reference.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

OUT = os.path.join(ROOT, "tests", "golden", "cube32_oracle_image.txt")


def main():
    import oracle
    import pgrec
    from make_cloud128_reference import trace_checksum

    sc = pgrec.CUBE_CONST
    rec = pgrec.trace(sc)
    ref = oracle.forward(rec, rec["first"], rec["bg"], sc.spp, sc.width, sc.height, sc.k, sc.iters)
    with open(OUT, "w") as f:
        f.write(f"# FP64 oracle image of {sc.name} ({sc.width}x{sc.height}, {sc.spp} spp, k={sc.k}, "
                f"{sc.iters} sweeps, {rec['n']} vertices)\n")
        f.write("# written by tests/golden/make_cube32_reference.py (oracle/ only; inputs from the seeded recorder)\n")
        f.write(f"trace_sha256 {trace_checksum(rec)}\n")
        f.write("residuals " + " ".join(f"{r:.17g}" for r in ref["residuals"]) + "\n")
        for row in ref["image"]:
            f.write(" ".join(f"{v:.17g}" for v in row) + "\n")
    print(f"wrote {OUT}")


def load():
    """Parsed file: dict(trace_sha256, residuals, image)."""
    with open(OUT) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    return {"trace_sha256": lines[0].split()[1],
            "residuals": np.array([float(v) for v in lines[1].split()[1:]]),
            "image": np.array([[float(v) for v in ln.split()] for ln in lines[2:]])}


if __name__ == "__main__":
    main()
