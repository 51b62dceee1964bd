"""Static drift field and carrier drift (the paper's Fig. 2 static field and
its carrier transport, here without Garfield++: a constant-mobility drift
that feeds Eq. 1).

Static field (Sec. 3's electrostatic solution, the sigma -> infinity limit of
the relaxation): every node of a column sits at its electrode's potential,
the node charges are q = C_n phi, and the field is the bulk extension of
those charges (the same operator as the weighting field).

Drift: dx/dt = s mu E(x) (s = +1 holes, -1 electrons), explicit midpoint
(RK2) steps of dt on the trilinear interpolation of E on the grid (grid
points at (i hx, j hy, (k + 1/2) hz); x, y periodic; z clamped to the first
and last planes, as in Eq. 1).  A step records its midpoint and its
velocity, so that sum_m H(x_m) . v_m dt is the midpoint rule of the line
integral.  A carrier stops after the step that ends inside a column (lateral
distance to the axis below the radius, nearest periodic image) or outside
0 <= z <= Lz; later steps repeat its last position with zero velocity.
TEST INFRASTRUCTURE ONLY: see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np

from . import extend


def node_potentials(columns, phi_cols):
    return np.concatenate([np.full(c.n_sources, float(p)) for c, p in zip(columns, phi_cols)])


def static_charges(sol, phi_cols):
    """q = C_n phi for per-column electrode potentials."""
    return sol.fit["Cn"] @ node_potentials(sol.columns, phi_cols)


def static_field(sol, phi_cols):
    """E [3, Nx, Ny, Nz] (V/m) of the electrodes held at phi_cols."""
    q = static_charges(sol, phi_cols)
    return extend.field_subgrid(sol.grid, sol.lay.src, q[:, None])[0]


def interp(E, grid, p):
    """Trilinear interpolation of E [3, Nx, Ny, Nz] at p = (x, y, z)."""
    Nx, Ny, Nz = grid.Nx, grid.Ny, grid.Nz
    fx = p[0] * Nx / grid.Lx
    fy = p[1] * Ny / grid.Ly
    fz = min(max(p[2] * Nz / grid.Lz - 0.5, 0.0), Nz - 1.0)
    ix, iy = math.floor(fx), math.floor(fy)
    kz = min(int(math.floor(fz)), Nz - 2)
    wx, wy, wz = fx - ix, fy - iy, fz - kz
    i0, j0 = ix % Nx, iy % Ny
    i1, j1 = (i0 + 1) % Nx, (j0 + 1) % Ny
    out = np.empty(3)
    for c in range(3):
        e = E[c]
        v00 = (1 - wz) * e[i0, j0, kz] + wz * e[i0, j0, kz + 1]
        v01 = (1 - wz) * e[i0, j1, kz] + wz * e[i0, j1, kz + 1]
        v10 = (1 - wz) * e[i1, j0, kz] + wz * e[i1, j0, kz + 1]
        v11 = (1 - wz) * e[i1, j1, kz] + wz * e[i1, j1, kz + 1]
        out[c] = (1 - wx) * ((1 - wy) * v00 + wy * v01) + wx * ((1 - wy) * v10 + wy * v11)
    return out


def inside_column(grid, columns, p):
    for c in columns:
        dx = (p[0] - c.x + 0.5 * grid.Lx) % grid.Lx - 0.5 * grid.Lx
        dy = (p[1] - c.y + 0.5 * grid.Ly) % grid.Ly - 0.5 * grid.Ly
        if dx * dx + dy * dy < c.radius * c.radius and c.z0 <= p[2] <= c.z1:
            return True
    return False


def drift(E, grid, columns, x0, sign, mu, dt, n_steps):
    """Positions and velocities [n, n_steps] (x, y, z, vx, vy, vz) of carriers
    started at x0 [n, 3] with charge signs sign [n] and mobilities mu [n]."""
    x0 = np.atleast_2d(np.asarray(x0, dtype=float))
    n = len(x0)
    out = np.zeros((6, n, n_steps))
    for a in range(n):
        p = x0[a].copy()
        s = float(sign[a]) * float(mu[a])
        alive = True
        for m in range(n_steps):
            if not alive:
                out[:3, a, m] = p
                continue
            k1 = s * interp(E, grid, p)
            pm = p + 0.5 * dt * k1
            k2 = s * interp(E, grid, pm)
            out[:3, a, m] = pm
            out[3:, a, m] = k2
            p = p + dt * k2
            p[0] %= grid.Lx
            p[1] %= grid.Ly
            if p[2] < 0.0 or p[2] > grid.Lz or inside_column(grid, columns, p):
                alive = False
    out[0] %= grid.Lx
    out[1] %= grid.Ly
    return out
