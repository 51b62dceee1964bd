"""Writes c5_oracle_subgrid.txt: the FP64 oracle's field of the 5x5 pixel cell
(grid 192x192x384, 50 columns, 256 time samples) on a seeded 8 x 8 x 8
subgrid at 4 of the time samples, for the full-size GPU test of that
configuration.

Calls only the oracle and the seeded input generators.  One oracle setup at
this size (fit of 12,800 sources to 102,400 collocation points by QR, then
the 12,800-mode relaxation) takes tens of minutes and about 45 GB of host
memory, so the values are stored instead of recomputed by the test.

    python tests/golden/make_c5_fixture.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "c5_oracle_subgrid.txt")
SEED = 55


def subgrid_indices(grid, n_t, seed=SEED):
    """Seeded indices: 8 per axis (sorted, distinct) and 4 time samples that
    include the first (1 ps) and the last (10 ns)."""
    rng = np.random.default_rng(seed)
    ix = np.sort(rng.choice(grid.Nx, 8, replace=False))
    iy = np.sort(rng.choice(grid.Ny, 8, replace=False))
    iz = np.sort(rng.choice(grid.Nz, 8, replace=False))
    mid = np.sort(rng.choice(np.arange(1, n_t - 1), 2, replace=False))
    it = np.array([0, mid[0], mid[1], n_t - 1])
    return ix, iy, iz, it


def main():
    import workloads as W
    import oracle as O

    w = W.c5_large(n_tracks=1)
    ix, iy, iz, it = subgrid_indices(w.grid, len(w.times))
    t0 = time.time()
    sol = O.solve(w, times=w.times[it])
    t1 = time.time()
    H = sol.H_subgrid(None, ix, iy, iz)                # [4, 3, 8, 8, 8]
    t2 = time.time()
    with open(OUT, "w") as f:
        f.write("# FP64 oracle field W = -grad psi [V/m] of the 5x5 pixel cell (192x192x384, 50 columns,\n")
        f.write("# 256 log-spaced time samples 1 ps - 10 ns, seed 5) on a seeded subgrid; written by\n")
        f.write("# tests/golden/make_c5_fixture.py (oracle only).  Lines: 'H t comp i j k value' with t the\n")
        f.write("# time-sample index, i j k grid indices.\n")
        f.write(f"# oracle setup {t1 - t0:.0f} s, subgrid field {t2 - t1:.0f} s\n")
        f.write("ix " + " ".join(str(int(v)) for v in ix) + "\n")
        f.write("iy " + " ".join(str(int(v)) for v in iy) + "\n")
        f.write("iz " + " ".join(str(int(v)) for v in iz) + "\n")
        f.write("it " + " ".join(str(int(v)) for v in it) + "\n")
        f.write(f"boundary_residual {O.fit.boundary_residual(sol.P, sol.S, sol.fit['F'], sol.fit['offset'], sol.phi_dc):.6e}\n")
        for a, t in enumerate(it):
            for c in range(3):
                for i, gi in enumerate(ix):
                    for j, gj in enumerate(iy):
                        for k, gk in enumerate(iz):
                            f.write(f"H {int(t)} {c} {int(gi)} {int(gj)} {int(gk)} {H[a, c, i, j, k]:.17e}\n")
    print(f"wrote {OUT}: setup {t1 - t0:.0f} s, field {t2 - t1:.0f} s")


def load(path=OUT):
    """(ix, iy, iz, it, H[4, 3, 8, 8, 8]) from the fixture."""
    idx, vals = {}, {}
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            p = line.split()
            if p[0] in ("ix", "iy", "iz", "it"):
                idx[p[0]] = np.array([int(v) for v in p[1:]])
            elif p[0] == "H":
                vals[tuple(int(v) for v in p[1:6])] = float(p[6])
    ix, iy, iz, it = idx["ix"], idx["iy"], idx["iz"], idx["it"]
    H = np.empty((len(it), 3, len(ix), len(iy), len(iz)))
    for a, t in enumerate(it):
        for c in range(3):
            for i, gi in enumerate(ix):
                for j, gj in enumerate(iy):
                    for k, gk in enumerate(iz):
                        H[a, c, i, j, k] = vals[(int(t), c, int(gi), int(gj), int(gk))]
    return ix, iy, iz, it, H


if __name__ == "__main__":
    main()
