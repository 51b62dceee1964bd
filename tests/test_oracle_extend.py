"""Pins of the oracle's bulk extension (extend.py)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import extend, greens


@pytest.fixture(scope="module")
def c1():
    return O.solve(W.workload("c1"))


def _fft_eval(grid, F):
    """Evaluate Re sum_k F(k) exp(i k.x) on the grid with numpy's FFT: the
    mirror box is 2 Lz tall with 2 Nz points; the grid is offset by h_z/2."""
    kx, ky, kz, _ = greens.mode_sets(grid)
    mx = np.rint(kx * grid.Lx / (2 * math.pi)).astype(int) % grid.Nx
    my = np.rint(ky * grid.Ly / (2 * math.pi)).astype(int) % grid.Ny
    mzi = np.rint(kz * grid.Lz / math.pi).astype(int)
    nz2 = 2 * grid.Nz
    arr = np.zeros((grid.Nx, grid.Ny, nz2), dtype=complex)
    shift = np.exp(1j * math.pi * mzi / nz2)            # z_k = (k + 1/2) h
    arr[np.ix_(mx, my, mzi % nz2)] = F * shift[None, None, :]
    out = np.fft.ifftn(arr) * arr.size
    return np.real(out[:, :, :grid.Nz])


def test_grid_sums_match_numpy_fft(c1):
    s = c1
    kx, ky, kz, vol = greens.mode_sets(s.grid)
    ti = [5, 40]
    H = s.H_subgrid(t_idx=ti)
    for n, t in enumerate(ti):
        rh = extend.rho_hat(s.grid, s.lay.src, s.q[:, t])[0]
        for a, k in enumerate((kx[:, None, None], ky[None, :, None], kz[None, None, :])):
            F = -1j * k * rh * greens.inv_k2(kx, ky, kz) / (greens.eps_abs(s.grid) * vol)
            ref = _fft_eval(s.grid, F)
            assert np.abs(H[n, a] - ref).max() < 1e-12 * np.abs(ref).max()


def test_field_is_lateral_curl_free(c1):
    """d W_y/dx = d W_x/dy, by spectral differentiation of the grid output."""
    s = c1
    H = s.H_subgrid(t_idx=[30])[0]
    g = s.grid
    kx = 2 * math.pi * np.fft.fftfreq(g.Nx, g.Lx / g.Nx)
    ky = 2 * math.pi * np.fft.fftfreq(g.Ny, g.Ly / g.Ny)
    dWy_dx = np.real(np.fft.ifft(1j * kx[:, None, None] * np.fft.fft(H[1], axis=0), axis=0))
    dWx_dy = np.real(np.fft.ifft(1j * ky[None, :, None] * np.fft.fft(H[0], axis=1), axis=1))
    assert np.abs(dWy_dx - dWx_dy).max() < 1e-10 * np.abs(dWx_dy).max()


def test_field_is_minus_gradient_of_potential(c1):
    s = c1
    p = np.array([[13.1e-6, 41.0e-6, 37.2e-6]])
    q = s.q[:, 20]
    W3 = extend.field_points(s.grid, s.lay.src, q, p)[0, 0]
    h = 1e-9
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        up = extend.field_points(s.grid, s.lay.src, q, p + e, comps=(3,))[0, 0, 0]
        dn = extend.field_points(s.grid, s.lay.src, q, p - e, comps=(3,))[0, 0, 0]
        assert abs(-(up - dn) / (2 * h) - W3[a]) < 1e-5 * np.abs(W3).max()


def test_single_cell_reflection_symmetry(c1):
    """Readout at the centre, bias at the corner: x -> -x maps the cell to
    itself, so W_x is odd and W_y, W_z are even; same for x <-> y."""
    H = c1.H_subgrid(t_idx=[10, 63])
    refl = np.concatenate([[0], np.arange(c1.grid.Nx - 1, 0, -1)])
    sc = np.abs(H).max()
    assert np.abs(H[:, 0] + H[:, 0][:, refl]).max() < 1e-10 * sc
    assert np.abs(H[:, 1] - H[:, 1][:, refl]).max() < 1e-10 * sc
    assert np.abs(H[:, 2] - H[:, 2][:, refl]).max() < 1e-10 * sc
    assert np.abs(H[:, 0] - H[:, 1].transpose(0, 2, 1, 3)).max() < 1e-10 * sc


def test_late_time_field_is_static_ramo_field(c1):
    """tau_1 = 1/mu_1 ~ 40 ps << 10 ns: the last sample equals the DC field."""
    s = c1
    Hl = s.H_subgrid(t_idx=[63])[0]
    Hi = extend.field_subgrid(s.grid, s.lay.src, s.rel["q_inf"])[0]
    assert np.abs(Hl - Hi).max() < 1e-12 * np.abs(Hi).max()


def test_potential_differences_match_ewald_far_from_sources():
    """Away from the columns the band-limited potential approaches the exact
    periodic (Ewald) potential of the same charges and their images."""
    w = W.tiny_cell(nx=16, nz=32, n_t=4, radius=8e-6)
    s = O.solve(w)
    g = s.grid
    q = s.rel["q_inf"]
    pts = np.array([[10e-6, 40e-6, 30e-6], [44e-6, 12e-6, 70e-6], [20e-6, 20e-6, 50e-6]])
    psi = extend.field_points(g, s.lay.src, q, pts, comps=(3,))[0, :, 0]
    eps = greens.eps_abs(g)
    box = (g.Lx, g.Ly, 2 * g.Lz)
    src = s.lay.src
    img = src * np.array([1.0, 1.0, -1.0])
    ref = np.array([sum(q[j] * (greens.ewald_green(box, [p - src[j]], eps)[0]
                                + greens.ewald_green(box, [p - img[j]], eps)[0])
                        for j in range(len(q))) for p in pts])
    d_bl = psi - psi[0]
    d_ex = ref - ref[0]
    assert np.abs(d_bl - d_ex).max() < 0.03 * np.abs(d_ex).max()
