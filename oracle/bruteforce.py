"""Brute-force finite-difference model of the same sensor (a consistency
check of the method, not a parity reference).

The column conductors are voxelised as in the paper's workflow (Sec. 2: the
geometry is voxelised on the regular grid): every voxel whose centre lies
within the column radius of its axis (periodic lateral distance) belongs to
the column, one equipotential node per grid layer.  The capacitance of the
nodes comes from the 7-point finite-difference Laplacian (periodic in x and
y, Neumann in z), eliminating the charge-free bulk voxels by a Schur
complement (sparse LU).  The resistive lines are the same as in
``geometry.resistive_line`` with one node per layer, so the relaxation uses
``relax.relax`` unchanged.

Against the spectral fit this model differs in discretisation (voxel
staircase vs band-limited point sources), so only loose agreement is
expected: parity unpinned for this comparison.  Its parts are pinned on their
own (tests/test_oracle_bruteforce.py): the operator's spectrum against the
closed form, a plane-filling column against parallel plates, and the Schur
complement against the charge of the harmonic extension solved densely.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .greens import eps_abs


def _laplacian(grid):
    """-Delta_h on the voxel grid (periodic x, y; Neumann z), sparse N x N."""
    nx, ny, nz = grid.Nx, grid.Ny, grid.Nz
    hx, hy, hz = grid.Lx / nx, grid.Ly / ny, grid.Lz / nz

    def idx(i, j, k):
        return (i * ny + j) * nz + k

    rows, cols, vals = [], [], []
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    c = idx(I, J, K)
    diag = np.zeros(c.size)
    for (di, dj, h) in ((1, 0, hx), (0, 1, hy)):
        for s in (1, -1):
            nb = idx((I + s * di) % nx, (J + s * dj) % ny, K)
            rows.append(c)
            cols.append(nb)
            vals.append(np.full(c.size, -1.0 / h ** 2))
            diag += 1.0 / h ** 2
    for s in (1, -1):
        ok = (K + s >= 0) & (K + s < nz)          # Neumann: no flux through z = 0, Lz
        rows.append(c[ok])
        cols.append(idx(I[ok], J[ok], K[ok] + s))
        vals.append(np.full(ok.sum(), -1.0 / hz ** 2))
        diag[ok] += 1.0 / hz ** 2
    rows.append(c)
    cols.append(c)
    vals.append(diag)
    n = nx * ny * nz
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def conductor_nodes(grid, columns):
    """Voxel -> node map: node = (column, layer) for voxels inside a column."""
    nx, ny, nz = grid.Nx, grid.Ny, grid.Nz
    hx, hy, hz = grid.Lx / nx, grid.Ly / ny, grid.Lz / nz
    x = np.arange(nx) * hx
    y = np.arange(ny) * hy
    z = (np.arange(nz) + 0.5) * hz
    node = -np.ones(nx * ny * nz, dtype=np.int64)
    off = 0
    for c in columns:
        if c.n_sources != nz or c.z0 != 0.0 or abs(c.z1 - grid.Lz) > 1e-15 * grid.Lz:
            raise ValueError("brute-force model needs full-height columns with one node per layer")
        dx = x[:, None] - c.x
        dy = y[None, :] - c.y
        dx -= grid.Lx * np.round(dx / grid.Lx)
        dy -= grid.Ly * np.round(dy / grid.Ly)
        inside = np.hypot(dx, dy) <= c.radius
        ii, jj = np.nonzero(inside)
        if ii.size == 0:
            raise ValueError("column thinner than the grid")
        for k in range(nz):
            node[(ii * ny + jj) * nz + k] = off + k
        off += nz
    return node, off


def node_capacitance(grid, columns):
    """C_nodes (n_nodes x n_nodes): node charges from node potentials, with the
    bulk voxels charge-free (Schur complement of eps V (-Delta_h))."""
    eps = eps_abs(grid)
    vol = grid.Lx * grid.Ly * grid.Lz / (grid.Nx * grid.Ny * grid.Nz)
    C = _laplacian(grid) * (eps * vol)
    node, n_nodes = conductor_nodes(grid, columns)
    cset = np.nonzero(node >= 0)[0]
    bset = np.nonzero(node < 0)[0]
    P = sp.csr_matrix((np.ones(cset.size), (np.arange(cset.size), node[cset])), shape=(cset.size, n_nodes))
    Ccc = C[cset][:, cset]
    if bset.size == 0:                                 # conductors fill the grid: nothing to eliminate
        X = np.zeros((0, n_nodes))
        Cn = P.T @ (Ccc @ P).toarray()
        Cn = 0.5 * (Cn + Cn.T)
        return np.asarray(Cn), {"X": X, "bset": bset, "cset": cset, "node": node}
    Ccb = C[cset][:, bset]
    Cbb = C[bset][:, bset].tocsc()
    Cbc_P = (C[bset][:, cset] @ P).toarray()
    X = spla.splu(Cbb).solve(Cbc_P)                    # bulk potentials per unit node potential
    Cn = P.T @ (Ccc @ P).toarray() - P.T @ (Ccb @ X)
    Cn = 0.5 * (Cn + Cn.T)
    return np.asarray(Cn), {"X": X, "bset": bset, "cset": cset, "node": node}


def bulk_potential(grid, columns, phi_nodes):
    """Potential on every voxel for node potentials phi (bulk charge-free)."""
    Cn, aux = node_capacitance(grid, columns)
    psi = np.empty(grid.Nx * grid.Ny * grid.Nz)
    psi[aux["cset"]] = phi_nodes[aux["node"][aux["cset"]]]
    psi[aux["bset"]] = -aux["X"] @ phi_nodes
    return psi.reshape(grid.Nx, grid.Ny, grid.Nz)
