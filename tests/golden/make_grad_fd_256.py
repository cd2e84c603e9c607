"""Writes grad_fd_256x512.json: oracle central differences for the gradient workload.

Sec. 4.2 differentiates the Sinkhorn divergence S (eq. sinkhorn-divergence) with respect to
the source measure p.  The stored values are directional derivatives <dS/dp, delta_k> of S
after exactly T = 400 iterations of Alg. 1 (no early stop), by central differences with the
relative step h = 1e-6 on the FP64 oracle (oracle.gradient.fd_directional), at the
256 x 512 Gauss-Legendre grid (L = 255), t = 1e-3 (eps = 4t, Sec. 3.2), balanced.
Inputs: pair 0 of a batch of 16 i.i.d. U(0,1) pairs normalised to unit mass (the runtime
experiment's fields of Sec. 4.1, inputs recipe "paper_uniform", base seed 4256); directions
from inputs.fd_directions (delta = p xi, xi ~ N(0,1), mass-preserving, ||delta||_a = ||p||_a).
Only oracle/ and the seeded input generators run here; nothing from the CUDA path.

    python tests/golden/make_grad_fd_256.py      # about 5 minutes of one CPU
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.grid import Grid  # noqa: E402
from oracle.gradient import fd_directional  # noqa: E402
from oracle.sinkhorn import divergence  # noqa: E402
from paper_2605_18389_gb300 import inputs  # noqa: E402

NLAT, T_HEAT, T_ITERS, H = 256, 1e-3, 400, 1e-6
EPS = 4.0 * T_HEAT
RECIPE, SEED, NPAIRS, PAIR = "paper_uniform", 4256, 16, 0
NDIRS, DIR_SEED = 3, 4257
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grad_fd_256x512.json")


def main():
    t0 = time.time()
    og = Grid(NLAT)
    p, q = inputs.pairs(RECIPE, SEED, NPAIRS, og.x, og.nlon, og.a_ring)
    p0, q0 = p[PAIR], q[PAIR]
    dirs = inputs.fd_directions(p0, og.a, NDIRS, DIR_SEED, balanced=True)
    ref = divergence(og, p0[None], q0[None], EPS, math.inf, T_ITERS, 0.0, 0, "l2", "sht")
    assert np.all(ref["status"] >= 0), ref["status"]
    fd = fd_directional(og, p0, q0, EPS, math.inf, T_ITERS, dirs, h=H)
    rec = {
        "what": "central differences of S after T iterations of Alg. 1 along delta_k (FP64 oracle)",
        "cite": "Sec. 4.2 (gradient of S w.r.t. the source measure), Alg. 1, eq. sinkhorn-divergence",
        "script": "tests/golden/make_grad_fd_256.py",
        "nlat": NLAT, "nlon": og.nlon, "lmax": NLAT - 1, "t": T_HEAT, "eps": EPS, "T": T_ITERS, "h": H,
        "recipe": RECIPE, "seed": SEED, "npairs": NPAIRS, "pair": PAIR,
        "ndirs": NDIRS, "dir_seed": DIR_SEED,
        "S": float(ref["S"][0]), "fd": [float(v) for v in fd],
        "seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
