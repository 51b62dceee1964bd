"""Ramo-Shockley-Riegler convolution, Eq. 1:

    i(t) = -(q / V_w) int_0^t H(x(t'), t - t') . v(t') dt'.

H here is the stored field W(x, t) = -grad psi of the step response to V_w
at t = 0; the impulse response of Eq. 1 is its time derivative, so Eq. 1 is
applied as i = -(q/V_w) d/dt int_0^t W(x(t'), t - t') . v(t') dt'.  Discrete
form, track steps m' = 0 .. n_steps-1 of length dt, output times
tau_m = m dt, m = 0 .. n_out-1:

    Q(tau_m) = sum_{m' <= m, m' < n_steps} W(x_m', (m - m' + 1/2) dt) . v_m' dt
    i(tau_m) = -(q / V_w) (Q(tau_m) - Q(tau_{m-1})) / dt,   Q(tau_{-1}) = 0.

The midpoint lag makes the perfectly conducting limit reproduce the
instantaneous Shockley-Ramo current.  W between grid points: trilinear,
periodic in x and y, z clamped to [z_0, z_{Nz-1}].  W between time samples:
linear in t, with W(x, 0) = 0 below the first sample and W held constant after
the last one.
"""
from __future__ import annotations

import numpy as np


def interp_space(grid, H, pts):
    """H [nt, 3, Nx, Ny, Nz] at points pts [n, 3] -> [n, nt, 3] (trilinear)."""
    hx, hy, hz = grid.Lx / grid.Nx, grid.Ly / grid.Ny, grid.Lz / grid.Nz
    fx = pts[:, 0] / hx
    fy = pts[:, 1] / hy
    fz = np.clip(pts[:, 2] / hz - 0.5, 0.0, grid.Nz - 1)
    i0 = np.floor(fx).astype(int)
    j0 = np.floor(fy).astype(int)
    k0 = np.minimum(np.floor(fz).astype(int), grid.Nz - 2)
    wx, wy, wz = fx - i0, fy - j0, fz - k0
    out = np.zeros((len(pts), H.shape[0], 3))
    for di in (0, 1):
        ii = (i0 + di) % grid.Nx
        ax = wx if di else 1.0 - wx
        for dj in (0, 1):
            jj = (j0 + dj) % grid.Ny
            ay = wy if dj else 1.0 - wy
            for dk in (0, 1):
                kk = k0 + dk
                az = wz if dk else 1.0 - wz
                w = ax * ay * az
                out += w[:, None, None] * H[:, :, ii, jj, kk].transpose(2, 0, 1)
    return out


def interp_time(times, Wt, lag):
    """Wt [n, nt, 3] (values at the time samples) at lags [n] -> [n, 3]."""
    t0, t1 = times[0], times[-1]
    out = np.empty((len(lag), 3))
    for n, s in enumerate(lag):
        if s <= t0:
            out[n] = Wt[n, 0] * (s / t0)
        elif s >= t1:
            out[n] = Wt[n, -1]
        else:
            j = np.searchsorted(times, s, side="right") - 1
            f = (s - times[j]) / (times[j + 1] - times[j])
            out[n] = (1.0 - f) * Wt[n, j] + f * Wt[n, j + 1]
    return out


def currents(grid, times, H, tracks, v_w=1.0, n_out=None, track_ids=None):
    """i [n_tracks_sel, n_out] for the selected tracks (all by default)."""
    dt = tracks.dt
    n_steps = tracks.n_steps
    n_out = tracks.n_out if n_out is None else n_out
    ids = np.arange(tracks.n_tracks) if track_ids is None else np.asarray(track_ids)
    out = np.zeros((len(ids), n_out))
    for r, tr in enumerate(ids):
        pos = np.stack([tracks.x[tr], tracks.y[tr], tracks.z[tr]], 1)
        vel = np.stack([tracks.vx[tr], tracks.vy[tr], tracks.vz[tr]], 1)
        Wt = interp_space(grid, H, pos)                       # [n_steps, nt, 3]
        Q = np.zeros(n_out)
        for m in range(n_out):
            mp = np.arange(min(m + 1, n_steps))
            lag = (m - mp + 0.5) * dt
            Wl = interp_time(times, Wt[mp], lag)
            Q[m] = np.sum(Wl * vel[mp]) * dt
        dQ = np.diff(np.concatenate([[0.0], Q]))
        out[r] = -(tracks.charge[tr] / v_w) * dQ / dt
    return out
