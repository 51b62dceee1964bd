"""Sensor geometry: point sources, collocation points, boundary targets and the
resistive line of each graphitised column.

Sources (Sec. 3: "point charges ... adjusted, in magnitude, to enforce the
boundary conditions"): M_c point charges on the axis of column c, at heights
z0 + (j + 1/2) Delta_c, Delta_c = (z1 - z0) / M_c, j = 0 .. M_c - 1 (bottom
first).  Columns are ordered as given; source index = offset(c) + j.

Collocation points: n_h * M_c heights z0 + (p + 1/2) (z1 - z0) / (n_h M_c)
times n_az azimuths theta_a = az0 + 2 pi a / n_az on the column surface
r = r_c, az0 = 0 by default.  (Other offsets are allowed; at az0 = pi/4 the
single-cell fit becomes ill-conditioned because the band-limited kernel of a
column's own sources nearly vanishes for one axial pattern there.)
Row index = offset(c) + (a * n_h * M_c + p).

Boundary target S phi: the column potential at a collocation height, linearly
interpolated between the node potentials at the source heights and held
constant beyond the end nodes.

Resistive line (Sec. 5: R = 4 rho L / (pi d^2), i.e. a conductance
pi r^2 / (rho * length)): neighbouring nodes are joined by
G_seg = pi r^2 / (rho Delta); the terminal end node sits Delta/2 from the
terminal, G_term = 2 G_seg, and the far end is open.  With node potentials
phi and terminal potentials V_T (V_w on the driven readout, 0 elsewhere):

    d q_j / dt = (K phi + b)_j,   b = G_term V_T at terminal nodes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Layout:
    src: np.ndarray          # [Ns, 3]
    src_col: np.ndarray      # [Ns] column index
    col_off: np.ndarray      # [n_col + 1] source offsets
    colloc: np.ndarray       # [Nc, 3]
    colloc_col: np.ndarray   # [Nc]
    colloc_z: np.ndarray     # [Nc] height
    colloc_off: np.ndarray   # [n_col + 1]

    @property
    def n_src(self):
        return len(self.src)


def validate(grid, columns):
    if grid.Nx % 2 or grid.Ny % 2:
        raise ValueError("Nx, Ny must be even")
    for c in columns:
        if not (0.0 <= c.z0 < c.z1 <= grid.Lz):
            raise ValueError("column z range outside the sensor")
        if c.radius <= 0 or c.resistivity < 0 or c.n_sources < 1:
            raise ValueError("bad column")
    n = len(columns)
    for i in range(n):
        for j in range(i + 1, n):
            dx = columns[i].x - columns[j].x
            dy = columns[i].y - columns[j].y
            dx -= grid.Lx * round(dx / grid.Lx)
            dy -= grid.Ly * round(dy / grid.Ly)
            if math.hypot(dx, dy) <= columns[i].radius + columns[j].radius:
                raise ValueError("overlapping columns")


def default_az0(n_az, az0):
    return 0.0 if az0 is None else az0


def layout(grid, columns, n_az=4, n_h=2, az0=None) -> Layout:
    validate(grid, columns)
    src, src_col, col_off = [], [], [0]
    colloc, colloc_col, colloc_z, colloc_off = [], [], [], [0]
    for ci, c in enumerate(columns):
        m = c.n_sources
        dz = (c.z1 - c.z0) / m
        zs = c.z0 + (np.arange(m) + 0.5) * dz
        src.append(np.stack([np.full(m, c.x), np.full(m, c.y), zs], 1))
        src_col.append(np.full(m, ci))
        col_off.append(col_off[-1] + m)
        nh = n_h * m
        zc = c.z0 + (np.arange(nh) + 0.5) * (c.z1 - c.z0) / nh
        for a in range(n_az):
            th = default_az0(n_az, az0) + 2.0 * math.pi * a / n_az
            colloc.append(np.stack([np.full(nh, c.x + c.radius * math.cos(th)),
                                    np.full(nh, c.y + c.radius * math.sin(th)), zc], 1))
            colloc_col.append(np.full(nh, ci))
            colloc_z.append(zc)
        colloc_off.append(colloc_off[-1] + n_az * nh)
    return Layout(np.concatenate(src), np.concatenate(src_col), np.array(col_off),
                  np.concatenate(colloc), np.concatenate(colloc_col), np.concatenate(colloc_z),
                  np.array(colloc_off))


def ring_sources(columns, lay: Layout, n_ring, frac=0.5, az0=0.0, n_az=4):
    """Sources on a ring of n_ring lines inside each column (a reading of the point charges "at the
    boundaries" of the active volume, Sec. 3, that resolves the azimuthal variation of the column
    potential which one axial line cannot): at every node height of the column, n_ring point
    sources at radius frac * r_c and azimuths az0 + 2 pi k / n_ring.  n_ring = 1 gives the axial
    sources of ``layout`` (frac ignored).  The ring's azimuthal harmonics must be resolved by the
    n_az collocation azimuths, so n_ring < n_az (n_ring = n_az leaves patterns that vanish at every
    collocation point and makes the fit singular).  Returns (src [Ns', 3], node [Ns']): the
    positions and, for each source, the node (column, height) whose potential it carries."""
    if n_ring < 1:
        raise ValueError("n_ring must be at least 1")
    if n_ring > 1 and n_ring >= n_az:
        raise ValueError("a ring needs fewer lines than collocation azimuths (n_ring < n_az)")
    if n_ring > 1 and not (0.0 < frac < 1.0):
        raise ValueError("the ring radius must lie inside the column (0 < frac < 1)")
    src, node = [], []
    for ci, c in enumerate(columns):
        m = c.n_sources
        zs = c.z0 + (np.arange(m) + 0.5) * (c.z1 - c.z0) / m
        rr = frac * c.radius if n_ring > 1 else 0.0
        for j in range(m):
            for k in range(n_ring):
                th = az0 + 2.0 * math.pi * k / n_ring
                src.append([c.x + rr * math.cos(th), c.y + rr * math.sin(th), zs[j]])
                node.append(lay.col_off[ci] + j)
    return np.array(src), np.array(node)


def interp_matrix(columns, lay: Layout):
    """S [Nc, Ns]: column potential at each collocation height from node potentials."""
    S = np.zeros((len(lay.colloc), lay.n_src))
    for i in range(len(lay.colloc)):
        c = lay.colloc_col[i]
        col = columns[c]
        m = col.n_sources
        dz = (col.z1 - col.z0) / m
        off = lay.col_off[c]
        u = (lay.colloc_z[i] - col.z0) / dz - 0.5        # fractional node index
        if u <= 0.0:
            S[i, off] = 1.0
        elif u >= m - 1:
            S[i, off + m - 1] = 1.0
        else:
            j = int(math.floor(u))
            f = u - j
            S[i, off + j] = 1.0 - f
            S[i, off + j + 1] = f
    return S


def node_resistivities(c):
    """Resistivity of each node's cell: the column's profile (Sec. 5's
    depth-dependent conductivity), else its uniform value."""
    if getattr(c, "rho_profile", None) is not None:
        rho = np.asarray(c.rho_profile, dtype=float)
        if rho.shape != (c.n_sources,):
            raise ValueError("rho_profile needs one value per source node")
        return rho
    return np.full(c.n_sources, float(c.resistivity))


def resistive_line(columns, lay: Layout, v_w=1.0):
    """K [Ns, Ns] and b [Ns] of the resistive columns.  Node j is the centre
    of a cell of height dz with resistivity rho_j; two neighbouring nodes are
    joined through two half cells, R = (rho_j + rho_j+1) dz / (2 pi r^2), and
    the terminal node reaches the electrode end through half a cell,
    R = rho_t dz / (2 pi r^2).  For a uniform column these are the segment
    conductance pi r^2 / (rho dz) of Sec. 5's R = 4 rho L / (pi d^2) and twice
    it at the terminal."""
    n = lay.n_src
    K = np.zeros((n, n))
    b = np.zeros(n)
    for ci, c in enumerate(columns):
        m = c.n_sources
        dz = (c.z1 - c.z0) / m
        off = lay.col_off[ci]
        rho = node_resistivities(c)
        area = math.pi * c.radius ** 2
        for j in range(m - 1):
            g = area / (0.5 * (rho[j] + rho[j + 1]) * dz)
            p, q = off + j, off + j + 1
            K[p, p] -= g
            K[q, q] -= g
            K[p, q] += g
            K[q, p] += g
        jl = m - 1 if c.terminal_top else 0
        gt = area / (0.5 * rho[jl] * dz)
        jt = off + jl
        K[jt, jt] -= gt
        b[jt] += gt * (v_w if c.driven else 0.0)
    return K, b


def phi_dc(columns, lay: Layout, v_w=1.0):
    """Late-time node potentials: V_w on the driven column, 0 elsewhere."""
    phi = np.zeros(lay.n_src)
    for ci, c in enumerate(columns):
        if c.driven:
            phi[lay.col_off[ci]:lay.col_off[ci + 1]] = v_w
    return phi


def column_resistance(c):
    """End-to-end resistance of a column, R = 4 rho L / (pi d^2) (Sec. 5)."""
    d = 2.0 * c.radius
    return 4.0 * c.resistivity * (c.z1 - c.z0) / (math.pi * d * d)
