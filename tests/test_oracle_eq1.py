"""Pins of the oracle's Eq. 1 convolution (eq1.py)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import eq1, extend


def test_trilinear_is_exact_on_linear_fields():
    g = W.GridSpec(40e-6, 40e-6, 60e-6, 8, 8, 12)
    x, y, z = extend.grid_coords(g)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    f = 3.0 + 2.0 * Z / g.Lz
    H = np.stack([f, 2 * f, -f])[None]                       # [1, 3, Nx, Ny, Nz]
    pts = np.array([[3e-6, 7e-6, 20e-6], [39e-6, 1e-6, 33.3e-6]])
    got = eq1.interp_space(g, H, pts)[:, 0, :]
    fz = 3.0 + 2.0 * pts[:, 2] / g.Lz
    assert np.allclose(got, np.stack([fz, 2 * fz, -fz], 1), rtol=1e-13)
    # z is clamped to the first/last grid plane
    got = eq1.interp_space(g, H, np.array([[5e-6, 5e-6, 0.0]]))[0, 0, 0]
    assert abs(got - (3.0 + 2.0 * z[0] / g.Lz)) < 1e-13


def test_time_interpolation_hand_values():
    times = np.array([1.0, 2.0, 4.0])
    Wt = np.array([[[1.0, 0, 0], [3.0, 0, 0], [7.0, 0, 0]]] * 4)
    lag = np.array([0.5, 1.5, 3.0, 9.0])
    got = eq1.interp_time(times, Wt, lag)[:, 0]
    assert np.allclose(got, [0.5, 2.0, 5.0, 7.0])


@pytest.fixture(scope="module")
def c1_full():
    s = O.solve(W.workload("c1"))
    return s, s.H_full()


def _tracks(g, n, steps, rng, v=1e5):
    return W.configs.mip_tracks(g, n, steps, rng, speed=v)


def test_perfect_conductor_gives_shockley_ramo():
    w = W.configs.with_resistivity(W.workload("c1"), 1e-14)
    s = O.solve(w)
    H = s.H_full(t_idx=[0, 63])
    times = s.times[[0, 63]]
    tr = _tracks(s.grid, 3, 20, np.random.default_rng(1))
    i = eq1.currents(s.grid, times, H, tr)
    for k in range(3):
        pos = np.stack([tr.x[k], tr.y[k], tr.z[k]], 1)
        vel = np.stack([tr.vx[k], tr.vy[k], tr.vz[k]], 1)
        Wx = eq1.interp_space(s.grid, H, pos)[:, -1, :]
        ramo = -(tr.charge[k] / 1.0) * np.sum(Wx * vel, axis=1)
        assert np.allclose(i[k, :20], ramo, rtol=1e-12, atol=1e-12 * np.abs(ramo).max())
        assert np.abs(i[k, 20:]).max() < 1e-12 * np.abs(ramo).max()


def test_stationary_carrier_and_linearity(c1_full):
    s, H = c1_full
    tr = _tracks(s.grid, 2, 10, np.random.default_rng(2))
    i1 = eq1.currents(s.grid, s.times, H, tr)
    tr.charge = tr.charge * -2.5
    i2 = eq1.currents(s.grid, s.times, H, tr)
    assert np.allclose(i2, -2.5 * i1, rtol=1e-13, atol=1e-30)
    for a in ("vx", "vy", "vz"):
        setattr(tr, a, np.zeros_like(getattr(tr, a)))
    assert np.abs(eq1.currents(s.grid, s.times, H, tr)).max() == 0.0


def _line_track(p0, p1, n_steps, dt, n_out):
    p0, p1 = np.asarray(p0), np.asarray(p1)
    v = (p1 - p0) / (n_steps * dt)
    steps = np.arange(n_steps)[None, :, None]
    pos = p0[None, None, :] + v[None, None, :] * dt * steps
    vel = np.broadcast_to(v, pos.shape)
    return W.TrackSet(pos[..., 0], pos[..., 1], pos[..., 2], vel[..., 0].copy(), vel[..., 1].copy(),
                      vel[..., 2].copy(), dt, np.array([1.0]), n_out)


def test_ramo_total_charge(c1_full):
    """Integrated current over a window long past relaxation equals
    (q/V_w)(psi_inf(x_end) - psi_inf(x_start)) up to path quadrature and the
    trilinear interpolation error (paths kept > 3 grid spacings from the
    column surfaces)."""
    s, H = c1_full
    for p0, p1 in (([10e-6, 40e-6, 95e-6], [20e-6, 45e-6, 5e-6]),
                   ([45e-6, 12e-6, 8e-6], [38e-6, 9e-6, 90e-6])):
        tr = _line_track(p0, p1, 200, 2.5e-11, 800)
        i = eq1.currents(s.grid, s.times, H, tr)
        psi = extend.field_points(s.grid, s.lay.src, s.rel["q_inf"], np.array([p0, p1]), comps=(3,))[0, :, 0]
        want = tr.charge[0] * (psi[1] - psi[0])
        got = np.sum(i[0]) * tr.dt
        assert abs(got - want) < 0.02 * abs(want)
