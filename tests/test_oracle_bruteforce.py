"""Consistency check of the reduced model against a brute-force finite-
difference model of the same sensor (voxelised columns, 7-point Laplacian,
Schur complement over the charge-free bulk).  The two discretisations differ,
so the bound is loose (20 %, the tolerance the comparison was planned with):
this is a physics consistency check, parity unpinned."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import bruteforce as BF, relax
from workloads.configs import UM


@pytest.fixture(scope="module")
def both():
    w = W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)
    sol = O.solve(w)
    Cbf, aux = BF.node_capacitance(w.grid, w.columns)
    return w, sol, Cbf, aux


def _colmat(C, nz):
    return np.array([[C[a * nz:(a + 1) * nz, b * nz:(b + 1) * nz].sum() for b in range(2)] for a in range(2)])


def test_bruteforce_is_self_consistent(both):
    w, sol, Cbf, aux = both
    assert np.abs(Cbf @ np.ones(len(Cbf))).max() < 1e-10 * np.abs(Cbf).max()      # neutral
    assert np.all(np.linalg.eigvalsh(Cbf)[1:] > 0)                                # PSD, one null vector
    psi = BF.bulk_potential(w.grid, w.columns, sol.phi_dc)
    lap = BF._laplacian(w.grid) @ psi.ravel()
    bulk = aux["bset"]
    assert np.abs(lap[bulk]).max() < 1e-9 * np.abs(lap).max()                     # charge-free bulk


def test_bruteforce_agrees_loosely_with_spectral_fit(both):
    w, sol, Cbf, aux = both
    nz = w.grid.Nz
    cm, cb = _colmat(sol.fit["Cn"], nz), _colmat(Cbf, nz)
    assert abs(cb[0, 0] / cm[0, 0] - 1) < 0.2
    r = relax.relax(Cbf, sol.K, sol.b, sol.phi_dc, w.times)
    assert abs(r["mu"][0] / sol.rel["mu"][0] - 1) < 0.2
    # DC potential at bulk voxels far from both columns (offsets removed)
    x, y, z = O.extend.grid_coords(w.grid)
    idx = [(4, 4, 8), (12, 3, 20), (3, 12, 27), (11, 12, 5)]
    pts = np.array([[x[i], y[j], z[k]] for i, j, k in idx])
    pm = O.extend.field_points(w.grid, sol.lay.src, sol.rel["q_inf"], pts, comps=(3,))[0, :, 0]
    psi = BF.bulk_potential(w.grid, w.columns, sol.phi_dc)
    pb = np.array([psi[i, j, k] for i, j, k in idx])
    pm, pb = pm - pm.mean(), pb - pb.mean()
    assert np.abs(pm - pb).max() < 0.2 * np.abs(pm).max()
