"""Pins of the depth-dependent column resistivity (Sec. 5 names a
depth-dependent conductivity profile as the next improvement): per-node
cells joined through half cells."""
import math
from dataclasses import replace

import numpy as np

import oracle as O
import workloads as W
from oracle import geometry


def _col_and_layout(profile=None, top=1):
    w = W.tiny_cell(nx=8, nz=16, n_t=6, m_req=12)
    cols = list(w.columns)
    cols[0] = replace(cols[0], terminal_top=top, rho_profile=profile)
    lay = geometry.layout(w.grid, cols, w.fit.n_az, w.fit.n_h, w.fit.az0)
    return w, cols, lay


def test_constant_profile_is_the_uniform_column():
    w, cols, lay = _col_and_layout()
    K0, b0 = geometry.resistive_line(cols, lay)
    c = cols[0]
    cols2 = list(cols)
    cols2[0] = replace(c, rho_profile=tuple([c.resistivity] * c.n_sources))
    K1, b1 = geometry.resistive_line(cols2, lay)
    assert np.array_equal(K0, K1) and np.array_equal(b0, b1)


def test_node_to_electrode_resistance_is_the_series_sum():
    """(-K)^-1 restricted to one column is the resistance matrix of a chain
    grounded at its terminal: node j sees the series sum of the half cells
    between it and the electrode end."""
    rng = np.random.default_rng(3)
    for top in (1, 0):
        w, cols, lay = _col_and_layout(top=top)
        c = cols[0]
        rho = rng.uniform(0.5, 3.0, c.n_sources) * c.resistivity
        cols[0] = replace(c, rho_profile=tuple(rho))
        K, _ = geometry.resistive_line(cols, lay)
        sl = slice(lay.col_off[0], lay.col_off[1])
        Rm = np.linalg.inv(-K[sl, sl])
        dz = (c.z1 - c.z0) / c.n_sources
        area = math.pi * c.radius ** 2
        m = c.n_sources
        order = list(range(m - 1, -1, -1)) if top else list(range(m))     # terminal first
        series = 0.0
        for k, j in enumerate(order):
            series += (rho[j] if k == 0 else 0.5 * (rho[j] + rho[order[k - 1]])) * dz / area
            if k == 0:
                series -= 0.5 * rho[j] * dz / area          # the terminal half cell only
            assert abs(Rm[j, j] - series) < 1e-12 * series, (top, j, Rm[j, j], series)


def test_uniform_column_resistance_matches_sec5_formula():
    """For a uniform column the far end sees R = 4 rho L / (pi d^2) less the
    half cell beyond the last node."""
    w, cols, lay = _col_and_layout()
    c = cols[0]
    K, _ = geometry.resistive_line(cols, lay)
    sl = slice(lay.col_off[0], lay.col_off[1])
    far = 0 if c.terminal_top else c.n_sources - 1
    R = np.linalg.inv(-K[sl, sl])[far, far]
    dz = (c.z1 - c.z0) / c.n_sources
    expect = geometry.column_resistance(c) - 0.5 * c.resistivity * dz / (math.pi * c.radius ** 2)
    assert abs(R - expect) < 1e-12 * expect


def test_more_resistive_far_half_slows_the_relaxation():
    """Raising the resistivity of the half of the readout column away from its
    terminal lowers the slowest relaxation rate."""
    w = W.tiny_cell(nx=8, nz=16, n_t=6, m_req=12)
    c = w.columns[0]
    m = c.n_sources
    prof = np.full(m, c.resistivity)
    far = slice(0, m // 2) if c.terminal_top else slice(m // 2, m)
    prof[far] *= 4.0
    w2 = replace(w, columns=[replace(c, rho_profile=tuple(prof))] + list(w.columns[1:]))
    mu0 = np.min(O.solve(w).rel["mu"])
    mu1 = np.min(O.solve(w2).rel["mu"])
    assert mu1 < mu0
