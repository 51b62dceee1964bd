"""Loss of Eq. 1 currents and its gradient by central finite differences
(FP64): the reference for the library's hand-written derivative.

L = mean over tracks and output times of i(tau_m)^2 (Eq. 1 currents with the
tracks' own charges; unit charges for normalised studies).  Parameters:

  0  s_R    resistivity scale of the readout columns (terminal at the top),
            rho_c -> s_R rho_c, derivative at s_R = 1;
  1  s_B    the same for the bias columns (terminal at the bottom);
  2  r      radius of every column [m];
  3  lambda lateral scale: Lx, Ly, column centres and the tracks' x, y, vx, vy
            scale by lambda (z, times and the source counts are fixed),
            derivative at lambda = 1; d/dpitch = d/dlambda / pitch.

Sec. 5 reads the time resolution's independence of the bias-electrode
diameter as the bias electrodes being practically irrelevant to the signal;
the test of this module checks the corresponding ordering of the gradients.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from .pipeline import solve
from . import eq1 as eq1mod

N_PARAMS = 4


def perturbed(w, tracks, k, eps):
    """Copies of (workload, tracks) with parameter k moved by eps (relative for
    the scales, absolute in metres for the radius)."""
    cols = list(w.columns)
    grid = w.grid
    tr = tracks
    if k == 0 or k == 1:
        want_top = 1 if k == 0 else 0
        cols = [replace(c, resistivity=c.resistivity * (1.0 + eps)) if c.terminal_top == want_top else c
                for c in cols]
    elif k == 2:
        cols = [replace(c, radius=c.radius + eps) for c in cols]
    elif k == 3:
        lam = 1.0 + eps
        grid = replace(grid, Lx=grid.Lx * lam, Ly=grid.Ly * lam)
        cols = [replace(c, x=c.x * lam, y=c.y * lam) for c in cols]
        tr = replace(tracks, x=tracks.x * lam, y=tracks.y * lam, vx=tracks.vx * lam, vy=tracks.vy * lam)
    return replace(w, grid=grid, columns=cols), tr


def loss(w, tracks):
    """(L, currents) for the workload and tracks, all in FP64."""
    sol = solve(w)
    H = sol.H_full()
    i = eq1mod.currents(sol.grid, sol.times, H, tracks, v_w=w.fit.v_w)
    return float(np.mean(i * i)), i


def fd_grad(w, tracks, rel_step=1e-4, params=range(N_PARAMS)):
    """Central-difference gradient of L for the listed parameters."""
    r0 = w.columns[0].radius
    g = np.full(N_PARAMS, np.nan)
    for k in params:
        h = rel_step * (r0 if k == 2 else 1.0)
        wp, tp = perturbed(w, tracks, k, +h)
        wm, tm = perturbed(w, tracks, k, -h)
        g[k] = (loss(wp, tp)[0] - loss(wm, tm)[0]) / (2.0 * h)
    return g


def fd_currents(w, tracks, rel_step=1e-4, params=range(N_PARAMS)):
    """Central-difference tangents of the currents, [N_PARAMS, n_tracks, n_out]
    (rows of parameters not listed are NaN): the reference for the library's
    forward-mode current tangents."""
    r0 = w.columns[0].radius
    out = None
    for k in params:
        h = rel_step * (r0 if k == 2 else 1.0)
        wp, tp = perturbed(w, tracks, k, +h)
        wm, tm = perturbed(w, tracks, k, -h)
        d = (loss(wp, tp)[1] - loss(wm, tm)[1]) / (2.0 * h)
        if out is None:
            out = np.full((N_PARAMS,) + d.shape, np.nan)
        out[k] = d
    return out
