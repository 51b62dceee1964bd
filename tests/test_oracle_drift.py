"""Pins of the oracle's static drift field and carrier drift."""
import math
from dataclasses import replace

import numpy as np

import oracle as O
import workloads as W
from oracle import drift as D, extend
from workloads.configs import UM


def _grid():
    return W.GridSpec(55 * UM, 55 * UM, 100 * UM, 8, 8, 16, 5.7)


def test_constant_field_gives_straight_lines():
    g = _grid()
    E = np.zeros((3, g.Nx, g.Ny, g.Nz))
    E[0], E[1], E[2] = 1e3, -2e3, 5e2
    dt, mu = 1e-12, 0.2
    x0 = np.array([[10 * UM, 20 * UM, 50 * UM]])
    out = D.drift(E, g, [], x0, [1.0], [mu], dt, 20)
    v = mu * np.array([1e3, -2e3, 5e2])
    for m in range(20):
        want = x0[0] + (m + 0.5) * dt * v
        want[:2] = np.mod(want[:2], [g.Lx, g.Ly])
        assert np.allclose(out[:3, 0, m], want, rtol=1e-12, atol=1e-18)
        assert np.allclose(out[3:, 0, m], v, rtol=1e-12)


def test_linear_field_converges_at_second_order():
    """E_z = a (z - zc) is reproduced exactly by the interpolation; the exact
    drift is z - zc = (z0 - zc) e^(s mu a t)."""
    g = _grid()
    a, zc, mu = 2e11, 50 * UM, 0.15
    zk = (np.arange(g.Nz) + 0.5) * g.Lz / g.Nz
    E = np.zeros((3, g.Nx, g.Ny, g.Nz))
    E[2] = a * (zk - zc)[None, None, :]
    z0, T = 58 * UM, 1e-10
    errs = []
    for n in (40, 80, 160):
        dt = T / n
        out = D.drift(E, g, [], np.array([[1 * UM, 1 * UM, z0]]), [-1.0], [mu], dt, n)
        z_end = out[2, 0, -1] + 0.5 * dt * out[5, 0, -1]          # midpoint + half step = end of the last step
        errs.append(abs(z_end - (zc + (z0 - zc) * math.exp(-mu * a * T))))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_carrier_stops_in_a_column():
    g = _grid()
    col = replace(W.tiny_cell(nx=8, nz=16).columns[0])
    E = np.zeros((3, g.Nx, g.Ny, g.Nz))
    E[0] = 1e4                                              # pushes holes towards +x
    x0 = np.array([[col.x - col.radius - 1 * UM, col.y, 50 * UM]])
    out = D.drift(E, g, [col], x0, [1.0], [0.2], 1e-10, 20)
    stopped = np.where(np.all(out[3:, 0, :] == 0.0, axis=0))[0]
    assert len(stopped) > 0
    m = stopped[0]
    assert np.hypot(out[0, 0, m] - col.x, out[1, 0, m] - col.y) < col.radius


def test_equal_electrode_potentials_give_no_field():
    w = W.tiny_cell(nx=8, nz=16, n_t=4)
    sol = O.solve(w)
    E1 = D.static_field(sol, [1.0, 1.0])
    E2 = D.static_field(sol, [1.0, 0.0])
    assert np.abs(E1).max() < 1e-9 * np.abs(E2).max()


def test_relaxation_reaches_the_static_charges():
    """Late in time the relaxing charges equal the static solution for the
    driven column at V_w and the others at zero."""
    w = W.tiny_cell(nx=8, nz=16, n_t=4)
    sol = O.solve(w, times=np.array([1e-12, 1e-9, 1e-3]))
    assert np.min(sol.rel["mu"]) * 1e-3 > 50
    q_static = D.static_charges(sol, [w.fit.v_w if c.driven else 0.0 for c in w.columns])
    assert np.linalg.norm(sol.q[:, -1] - q_static) < 1e-9 * np.linalg.norm(q_static)


def test_line_integral_of_the_field_is_the_potential_difference():
    """From the bias column's surface to the readout's, along the cell
    diagonal at mid-height, the integral of E . dl is the potential
    difference (within the thin-wire residual of the surface potential)."""
    w = W.tiny_cell(nx=32, nz=32, n_t=4, radius=5 * UM)
    sol = O.solve(w)
    ro, bi = w.columns
    q = D.static_charges(sol, [0.0, 1.0])                    # bias at 1 V, readout at 0
    a = np.array([bi.x, bi.y]); b = np.array([ro.x, ro.y])
    u = (b - a) / np.linalg.norm(b - a)
    s = np.linspace(bi.radius, np.linalg.norm(b - a) - ro.radius, 801)
    pts = np.array([[a[0] + t * u[0], a[1] + t * u[1], 0.5 * w.grid.Lz] for t in s])
    Ep = extend.field_points(w.grid, sol.lay.src, q, pts)[0]
    integral = np.trapezoid(Ep[:, 0] * u[0] + Ep[:, 1] * u[1], s)
    assert abs(integral - 1.0) < 0.03, integral
