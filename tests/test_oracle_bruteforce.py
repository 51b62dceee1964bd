"""Consistency check of the reduced model against a brute-force finite-
difference model of the same sensor (voxelised columns, 7-point Laplacian,
Schur complement over the charge-free bulk).  The two discretisations differ,
so the bound is loose (20 %, the tolerance the comparison was planned with):
this is a physics consistency check, parity unpinned.  The model's own pieces are pinned below:
the Laplacian's spectrum against its closed form, the node assembly against parallel plates, and
the Schur complement against its definition solved densely."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import bruteforce as BF, relax
from workloads.configs import UM, ColumnSpec, GridSpec
from oracle.greens import eps_abs


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


def _full_height(grid, x, y, radius):
    return ColumnSpec(x=x, y=y, z0=0.0, z1=grid.Lz, radius=radius, resistivity=1.0, terminal_top=1, driven=0,
                      n_sources=grid.Nz)


def test_laplacian_spectrum_is_the_closed_form():
    """-Delta_h on a 4 x 3 x 5 grid (periodic x, y; no flux through z = 0, Lz, cell-centred):
    eigenvalues (2 - 2 cos(2 pi i / n_x)) / h_x^2 + (2 - 2 cos(2 pi j / n_y)) / h_y^2
    + (2 - 2 cos(pi k / n_z)) / h_z^2."""
    g = GridSpec(40e-6, 30e-6, 50e-6, 4, 3, 5)
    hx, hy, hz = g.Lx / g.Nx, g.Ly / g.Ny, g.Lz / g.Nz
    got = np.sort(np.linalg.eigvalsh(BF._laplacian(g).toarray()))
    i, j, k = np.meshgrid(np.arange(g.Nx), np.arange(g.Ny), np.arange(g.Nz), indexing="ij")
    want = np.sort(((2 - 2 * np.cos(2 * np.pi * i / g.Nx)) / hx ** 2 + (2 - 2 * np.cos(2 * np.pi * j / g.Ny)) / hy ** 2
                    + (2 - 2 * np.cos(np.pi * k / g.Nz)) / hz ** 2).ravel())
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * want.max())


def test_plane_filling_column_is_a_stack_of_parallel_plates():
    """A column that covers the whole cross-section leaves no bulk: its layer nodes are parallel
    plates h_z apart, C = eps A / h_z times the no-flux second difference along z."""
    g = GridSpec(30e-6, 30e-6, 60e-6, 4, 4, 6)
    C, aux = BF.node_capacitance(g, [_full_height(g, 15e-6, 15e-6, 1.0)])
    assert aux["bset"].size == 0
    hz = g.Lz / g.Nz
    L = 2 * np.eye(g.Nz) - np.eye(g.Nz, k=1) - np.eye(g.Nz, k=-1)
    L[0, 0] = L[-1, -1] = 1
    want = eps_abs(g) * g.Lx * g.Ly / hz * L
    assert np.allclose(C, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_schur_complement_is_the_charge_of_the_harmonic_extension():
    """Node capacitance from its definition: for a unit potential on one node (zero on the others),
    solve the charge-free bulk densely, apply eps V (-Delta_h) and sum the charge on each node's
    voxels.  Two thin columns on a 6 x 6 x 4 grid."""
    g = GridSpec(30e-6, 30e-6, 20e-6, 6, 6, 4)
    cols = [_full_height(g, 10e-6, 10e-6, 5.5e-6), _full_height(g, 25e-6, 20e-6, 5.5e-6)]
    C, aux = BF.node_capacitance(g, cols)
    node, n_nodes = BF.conductor_nodes(g, cols)
    A = BF._laplacian(g).toarray() * eps_abs(g) * (g.Lx * g.Ly * g.Lz / (g.Nx * g.Ny * g.Nz))
    bulk = node < 0
    want = np.zeros((n_nodes, n_nodes))
    for a in range(n_nodes):
        psi = np.zeros(node.size)
        psi[node == a] = 1.0
        rhs = -A[np.ix_(bulk, ~bulk)] @ psi[~bulk]
        psi[bulk] = np.linalg.solve(A[np.ix_(bulk, bulk)], rhs)
        q = A @ psi
        assert np.abs(q[bulk]).max() < 1e-9 * np.abs(q).max()
        for b in range(n_nodes):
            want[b, a] = q[node == b].sum()
    assert np.allclose(C, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
