"""Pins of the oracle's ring of source lines (``geometry.ring_sources``, ``pipeline.solve(n_ring=)``):
the point charges placed on a ring inside each column rather than on its axis (Sec. 3 places them
at the boundaries of the active volume).  One line reproduces the axial sources; three lines
resolve the azimuthal variation of the column potential that one axial line leaves as boundary
error; the node capacitance keeps the Maxwell-matrix sign pattern, reciprocity and neutrality;
the source charges start at zero and follow the node potentials of the relaxation."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import geometry
from workloads.configs import UM, OHM_CM


@pytest.fixture(scope="module")
def cell():
    grid, cols = W.configs.pixel_matrix(3, 55 * UM, 200 * UM, 16, 32, 6 * UM, 0.1 * OHM_CM, 1.0 * OHM_CM, 16,
                                        np.random.default_rng(4))
    w = W.Workload("m3", grid, cols, W.FitSpec(), W.log_times(8))
    times = np.array([0.0, 1e-12, 1e-9, 1.0])
    return w, O.solve(w, times=times), O.solve(w, times=times, n_ring=3)


def _residual(s):
    return O.fit.boundary_residual(s.P, s.S, s.fit["F"], s.fit["offset"], s.phi_dc)


def _surface_error(s, cols):
    """DC potential on the column surfaces at points that are not collocation points (azimuths
    pi/4 + k pi/2, node heights), against the column potential there, after the free offset."""
    pts, tgt = [], []
    for ci, c in enumerate(cols):
        m = c.n_sources
        for j in range(1, m - 1):
            z = c.z0 + (j + 0.5) * (c.z1 - c.z0) / m
            for k in range(4):
                th = math.pi / 4 + k * math.pi / 2
                pts.append([c.x + c.radius * math.cos(th), c.y + c.radius * math.sin(th), z])
                tgt.append(s.phi_dc[s.lay.col_off[ci] + j])
    tgt = np.array(tgt)
    psi = O.extend.field_points(s.grid, s.sources, s.rel["q_inf"], np.array(pts), comps=(3,))[0, :, 0]
    d = psi - np.mean(psi - tgt) - tgt
    return np.linalg.norm(d) / np.linalg.norm(tgt)


def test_one_line_is_the_axial_layout(cell):
    w, axial, _ = cell
    src, node = geometry.ring_sources(w.columns, axial.lay, 1)
    assert np.array_equal(src, axial.lay.src)
    assert np.array_equal(node, np.arange(axial.lay.n_src))


def test_three_lines_cut_the_boundary_error(cell):
    w, axial, ring = cell
    assert ring.sources.shape[0] == 3 * axial.lay.n_src
    # at the collocation points
    assert _residual(axial) > 0.05
    assert _residual(ring) < 0.01
    # and between them, on the same surfaces
    assert _surface_error(ring, w.columns) < 0.3 * _surface_error(axial, w.columns)


def test_ring_capacitance_is_a_maxwell_matrix(cell):
    w, _, ring = cell
    Cn, off = ring.fit["Cn"], ring.lay.col_off
    n = len(w.columns)
    Cc = np.array([[Cn[off[a]:off[a + 1], off[b]:off[b + 1]].sum() for b in range(n)] for a in range(n)])
    assert np.all(np.diag(Cc) > 0)
    assert np.all(Cc[~np.eye(n, dtype=bool)] < 0)
    assert ring.fit["asymmetry"] < 1e-2                                  # reciprocity of N^T F
    assert np.abs(Cn.sum(1)).max() < 1e-9 * np.abs(Cn).max()           # neutral cell


def test_ring_charges_start_at_zero_and_follow_the_nodes(cell):
    w, _, ring = cell
    q = ring.q
    assert np.abs(q[:, 0]).max() < 1e-12 * np.abs(q[:, -1]).max()      # q(0) = 0
    assert np.allclose(q[:, -1], ring.rel["q_inf"], rtol=0, atol=1e-9 * np.abs(q[:, -1]).max())
    # the node charges the sources carry are the relaxation's node charges (to the symmetrisation)
    qn = ring.fit["N"].T @ q
    assert np.abs(qn - ring.rel["q_node"]).max() < 1e-3 * np.abs(ring.rel["q_node"]).max()


def test_aliased_ring_is_refused(cell):
    w, axial, _ = cell
    with pytest.raises(ValueError):
        geometry.ring_sources(w.columns, axial.lay, 4, n_az=4)
    with pytest.raises(ValueError):
        geometry.ring_sources(w.columns, axial.lay, 3, frac=1.2)


def test_residual_keeps_falling_with_more_lines(cell):
    """Five lines, with six collocation azimuths to resolve them, take the residual further down
    than three (the second azimuthal harmonic of the column potential becomes representable)."""
    w, _, ring3 = cell
    w6 = W.Workload("m3", w.grid, w.columns, W.FitSpec(n_az=6), w.times)
    ring5 = O.solve(w6, times=np.array([0.0, 1.0]), n_ring=5)
    assert ring5.sources.shape[0] == 5 * ring3.lay.n_src
    assert _residual(ring5) < 0.8 * _residual(ring3)
    assert ring5.fit["asymmetry"] < 1e-2
