"""Pins of the oracle's geometry and boundary fit (geometry.py, fit.py)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import geometry, greens, fit
from workloads.configs import pixel_matrix, UM, OHM_CM
from tests.golden.read import values


@pytest.fixture(scope="module")
def c1():
    return O.solve(W.workload("c1"), want_cond=True)


@pytest.fixture(scope="module")
def small3x3():
    rng = np.random.default_rng(2)
    grid, cols = pixel_matrix(3, 55 * UM, 100 * UM, 24, 32, 6 * UM, 0.1 * OHM_CM, 1 * OHM_CM, 32, rng)
    w = W.Workload("s3", grid, cols, W.FitSpec(), W.log_times(16))
    return O.solve(w)


def test_paper_resistance_formula():
    """Sec. 5: d = 12 um, L = 500 um, 0.75 Ohm cm -> R = 4 rho L/(pi d^2), 'about 30 kOhm'."""
    v = values("paper_sec5_column.txt")
    col = W.ColumnSpec(0, 0, 0, v["L_um"] * UM, v["d_um"] / 2 * UM, v["rho_ohm_cm"] * OHM_CM, 1, 1, 256)
    R = geometry.column_resistance(col)
    assert abs(R - 33157.3) < 1.0
    assert abs(R / (v["R_about_kohm"] * 1e3) - 1.0) < 0.15
    # the discrete line: terminal half-segment + (M-1) segments = (M - 1/2) Delta rho / (pi r^2)
    grid = W.GridSpec(55 * UM, 55 * UM, v["L_um"] * UM, 8, 8, 256)
    lay = geometry.layout(grid, [col])
    K, b = geometry.resistive_line([col], lay, 1.0)
    g = K[0, 1]
    gt = -K[-1, -1] - g
    r_series = 1.0 / gt + (col.n_sources - 1) / g
    assert abs(r_series / (R * (col.n_sources - 0.5) / col.n_sources) - 1.0) < 1e-12
    assert abs(b[-1] - gt * 1.0) < 1e-12 * gt


def test_fit_neutral_and_uniform_potential(c1):
    F = c1.fit["F"]
    s = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * s * F.shape[0]     # sum q = 0 for any phi
    assert np.abs(F @ np.ones(F.shape[1])).max() < 1e-12 * s * F.shape[0]  # uniform phi -> q = 0
    assert c1.fit["cond_A"] < 1e4


def test_fit_matches_lagrange_kkt(c1):
    """Independent route: the constrained least squares through its Lagrange
    (KKT) system, solved with numpy's dense solver after column scaling."""
    P, S = c1.P, c1.S
    nc, ns = P.shape
    A = np.hstack([P, np.ones((nc, 1))])
    d = 1.0 / np.linalg.norm(A, axis=0)
    As = A * d
    con = np.concatenate([np.ones(ns) * d[:ns], [0.0]])[None, :]
    M = np.block([[As.T @ As, con.T], [con, np.zeros((1, 1))]])
    rhs = np.vstack([As.T @ S, np.zeros((1, ns))])
    X = np.linalg.solve(M, rhs)[:ns + 1] * d[:, None]
    F2 = X[:ns]
    assert np.linalg.norm(F2 - c1.fit["F"]) < 1e-8 * np.linalg.norm(c1.fit["F"])


def test_capacitance_is_a_maxwell_matrix(small3x3):
    """Green reciprocity and the sign pattern of a Maxwell capacitance matrix."""
    s = small3x3
    assert s.fit["asymmetry"] < 1e-6
    off = s.lay.col_off
    n = len(s.columns)
    Cn = s.fit["Cn"]
    C = np.array([[Cn[off[i]:off[i + 1], off[j]:off[j + 1]].sum() for j in range(n)] for i in range(n)])
    scale = np.abs(C).max()
    assert np.allclose(C, C.T, atol=1e-10 * scale)
    assert np.all(np.diag(C) > 0)
    assert np.all(C[~np.eye(n, dtype=bool)] <= 1e-10 * scale)
    assert np.abs(C.sum(axis=1)).max() < 1e-10 * scale


def test_dc_boundary_values_between_collocation_points(c1):
    """The fitted DC charges hold the driven column at V_w and the bias column
    at 0 (up to the common offset) at surface points the fit never saw."""
    s = c1
    q = s.rel["q_inf"]
    c = s.fit["offset"] @ s.phi_dc
    pts = []
    for col in s.columns:
        for th in (0.3, 1.9):
            for z in (20e-6, 47.3e-6, 81e-6):
                pts.append([col.x + col.radius * math.cos(th), col.y + col.radius * math.sin(th), z])
    pts = np.array(pts)
    psi = O.extend.field_points(s.grid, s.lay.src, q, pts, comps=(3,))[0, :, 0]
    want = np.array([1.0] * 6 + [0.0] * 6) - c
    assert np.abs(psi - want).max() < 2e-2
    # and at the collocation points themselves the residual is rounding only
    assert O.fit.boundary_residual(s.P, s.S, s.fit["F"], s.fit["offset"], s.phi_dc) < 1e-10


def test_potential_matrix_agrees_with_spectral_extension(c1):
    """Two routes to the potential of the same charges: the fit matrix P
    (lateral table x cosine tables) and the extension (rho^ -> mode sum)."""
    s = c1
    rng = np.random.default_rng(3)
    q = rng.standard_normal(s.lay.n_src)
    q -= q.mean()
    idx = rng.choice(len(s.lay.colloc), 12, replace=False)
    a = (s.P @ q)[idx]
    b = O.extend.field_points(s.grid, s.lay.src, q, s.lay.colloc[idx], comps=(3,))[0, :, 0]
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10 * np.abs(a).max())


def test_geometry_rejects_overlap():
    grid = W.GridSpec(55 * UM, 55 * UM, 100 * UM, 8, 8, 16)
    a = W.ColumnSpec(10 * UM, 10 * UM, 0, 100 * UM, 5 * UM, 1e-3, 1, 1, 16)
    b = W.ColumnSpec(18 * UM, 10 * UM, 0, 100 * UM, 5 * UM, 1e-3, 0, 0, 16)
    with pytest.raises(ValueError):
        geometry.layout(grid, [a, b])
