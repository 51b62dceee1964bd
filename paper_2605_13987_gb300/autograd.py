"""torch.autograd.Function over the library's derivative of the Eq. 1 loss.

The design vector is theta = (s_R, s_B, dr, lam):
  s_R, s_B  scales of the readout / bias column resistivities,
  dr        radius offset added to every column [m],
  lam       lateral scale (Lx, Ly, column centres and the tracks' x, y,
            vx, vy scale together; z, times and source counts are fixed).
theta = (1, 1, 0, 1) is the design as given.  forward() builds the sensor
at theta, runs the fit (Sec. 3) and the relaxation (Sec. 5) and calls
wt_eq1_loss_grad, which returns L = mean i^2 (Eq. 1) and its derivative at
that design with respect to relative resistivity changes, absolute radius
change and relative lateral scale; backward() maps that to theta.  No
computation happens here: every step runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, replace as _replace
from types import SimpleNamespace

import numpy as np
import torch

from .sensor import Sensor

BASE_THETA = (1.0, 1.0, 0.0, 1.0)


def _copy(obj, **kw):
    try:
        return _replace(obj, **kw)
    except TypeError:
        d = dict(vars(obj))
        d.update(kw)
        return SimpleNamespace(**d)


def design_at(grid, columns, tracks, theta):
    """(grid, columns, tracks) of the design theta (host copies; the track
    dict may hold numpy arrays or torch tensors)."""
    sR, sB, dr, lam = (float(v) for v in theta)
    g = _copy(grid, Lx=grid.Lx * lam, Ly=grid.Ly * lam)
    cols = [_copy(c, x=c.x * lam, y=c.y * lam, radius=c.radius + dr,
                  resistivity=c.resistivity * (sR if int(c.terminal_top) else sB)) for c in columns]
    tr = dict(tracks)
    for k in ("x", "y", "vx", "vy"):
        tr[k] = tracks[k] * lam
    return g, cols, tr


@dataclass
class FitOptions:
    n_az: int = 4
    n_h: int = 2
    v_w: float = 1.0
    az0: float = 0.0


class Eq1Loss(torch.autograd.Function):
    """L(theta) with its hand-written gradient; see the module docstring."""

    @staticmethod
    def forward(ctx, theta, grid, columns, times, tracks, fit=None, device=0):
        th = theta.detach().to("cpu", torch.float64).numpy()
        fit = fit or FitOptions()
        g, cols, tr = design_at(grid, columns, tracks, th)
        sen = Sensor(g, cols, device)
        try:
            sen.fit(n_az=fit.n_az, n_h=fit.n_h, v_w=fit.v_w, az0=fit.az0)
            sen.relax(times)
            loss, d = sen.loss_grad(tr)
        finally:
            sen.close()
        # the library differentiates relative changes at the design itself
        dtheta = np.array([d[0] / th[0], d[1] / th[1], d[2], d[3] / th[3]])
        ctx.save_for_backward(torch.as_tensor(dtheta, dtype=theta.dtype, device=theta.device))
        return theta.new_tensor(loss)

    @staticmethod
    def backward(ctx, grad_out):
        (dtheta,) = ctx.saved_tensors
        return grad_out * dtheta, None, None, None, None, None, None


def eq1_loss(theta, grid, columns, times, tracks, fit=None, device=0):
    """Differentiable L(theta) (a 0-d tensor)."""
    return Eq1Loss.apply(theta, grid, columns, times, tracks, fit, device)
