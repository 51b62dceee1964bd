"""Object wrapper over the C ABI: one Sensor = one wt_ctx."""
from __future__ import annotations

import numpy as np

from . import _binding as B


def extend_batch(sensors, precision="fp32", outs=None, stream=None):
    """Bulk extension of several relaxed sensors in one captured launch sequence
    (wt_batch_run); returns the list of H tensors."""
    import torch
    prec = B.WT_FP64 if precision in ("fp64", B.WT_FP64) else B.WT_FP32
    if outs is None:
        dt = torch.float64 if prec == B.WT_FP64 else torch.float32
        outs = [torch.empty(s.h_shape(), dtype=dt, device=f"cuda:{s.device}") for s in sensors]
    B.wt_batch_run([s.ctx for s in sensors], prec, outs, stream)
    return outs


class Sensor:
    """Sensor(grid, columns, device=0); then fit() -> relax(times) -> extend()."""

    def __init__(self, grid, columns, device: int = 0):
        self.grid = grid
        self.columns = list(columns)
        self.device = device
        self.ctx = B.wt_create(grid, device)
        B.wt_add_columns(self.ctx, self.columns)
        for k, c in enumerate(self.columns):          # depth profiles carried by the column specs
            prof = getattr(c, "rho_profile", None)
            if prof is not None:
                B.wt_set_resistivity_profile(self.ctx, k, prof)
        self.n_sources = sum(int(c.n_sources) for c in self.columns)
        self.times = None

    def fit(self, n_az=4, n_h=2, tikhonov=0.0, v_w=1.0, az0=0.0, refine=0):
        return B.wt_fit(self.ctx, n_az, n_h, tikhonov, v_w, az0, refine)

    def relax(self, times):
        self.times = np.asarray(times, dtype=np.float64)
        B.wt_relax(self.ctx, self.times)

    def h_shape(self):
        g = self.grid
        return (len(self.times), 3, g.Nx, g.Ny, g.Nz)

    def extend(self, precision="fp32", out=None, stream=None):
        import torch
        prec = B.WT_FP64 if precision in ("fp64", B.WT_FP64) else B.WT_FP32
        if out is None:
            dt = torch.float64 if prec == B.WT_FP64 else torch.float32
            out = torch.empty(self.h_shape(), dtype=dt, device=f"cuda:{self.device}")
        B.wt_extend(self.ctx, prec, out, stream)
        return out

    def sample_H(self, xyz, times):
        return B.wt_sample_H(self.ctx, xyz, times)

    def eq1(self, H, tracks, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((int(tracks["n_tracks"]), int(tracks["n_out"])), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        B.wt_eq1(self.ctx, H, tracks, out, stream)
        return out

    def eq1_direct(self, tracks, out=None, stream=None):
        """Eq. 1 currents without writing H (from the field's rank-r form)."""
        import torch
        if out is None:
            out = torch.empty((int(tracks["n_tracks"]), int(tracks["n_out"])), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        B.wt_eq1_direct(self.ctx, tracks, out, stream)
        return out

    def loss(self, tracks, precision="fp32"):
        """Mean squared Eq. 1 current over tracks and output times."""
        prec = B.WT_FP64 if precision in ("fp64", B.WT_FP64) else B.WT_FP32
        return B.wt_eq1_loss(self.ctx, prec, tracks)

    def loss_grad(self, tracks):
        """(loss, dL/d[s_R, s_B, r, lambda]) by the library's tangent-linear derivative."""
        return B.wt_eq1_loss_grad(self.ctx, tracks)

    def set_resistivity_profile(self, column, rho):
        """Per-node resistivities of one column (None: uniform); takes effect at the next relax()."""
        B.wt_set_resistivity_profile(self.ctx, column, rho)

    def loss_grad_profile(self, tracks, delta):
        """(loss, dL/deps) along rho_j -> rho_j (1 + eps delta_j)."""
        return B.wt_eq1_loss_grad_profile(self.ctx, tracks, delta)

    def tangents(self, tracks):
        """(i, di, loss, grad): Eq. 1 currents [n_tracks, n_out] and their
        derivatives [4, n_tracks, n_out] along (s_R, s_B, r, lambda), device FP32."""
        import torch
        n_tr, n_out = int(tracks["n_tracks"]), int(tracks["n_out"])
        dev = f"cuda:{self.device}"
        i = torch.empty((n_tr, n_out), dtype=torch.float32, device=dev)
        di = torch.empty((4, n_tr, n_out), dtype=torch.float32, device=dev)
        loss, grad = B.wt_eq1_tangents(self.ctx, tracks, i, di)
        return i, di, loss, grad

    def features(self, x, dt, t0=0.0, dx=None, lo=0.1, hi=0.9, cfd=0.5, stream=None):
        """Signal features of device waveforms x [n_tracks, n] (and their
        derivatives along tangents dx [n_dir, n_tracks, n]): (f, df)."""
        return B.wt_features(self.ctx, x, t0, dt, lo, hi, cfd, dx=dx, stream=stream)

    def static_field(self, phi_cols, precision="fp32"):
        """Static field [3, Nx, Ny, Nz] of the electrodes held at phi_cols volts."""
        import torch
        prec = B.WT_FP64 if precision in ("fp64", B.WT_FP64) else B.WT_FP32
        g = self.grid
        E = torch.empty((3, g.Nx, g.Ny, g.Nz), dtype=torch.float64 if prec == B.WT_FP64 else torch.float32,
                        device=f"cuda:{self.device}")
        return B.wt_static_field(self.ctx, phi_cols, prec, E)

    def drift(self, E, x0, smu, n_steps, dt, charge=None):
        """Carrier tracks in the static field E (FP32): a track dict for eq1()."""
        import torch
        out = B.wt_drift(self.ctx, E, x0, smu, n_steps, dt)
        out.update(n_tracks=int(x0.shape[0]), n_steps=int(n_steps), n_out=2 * int(n_steps), dt=float(dt),
                   charge=1.0, q=charge)
        return out

    def shape(self, i, dt, tau, order, gain=1.0, noise=None, noise_rms=0.0, out=None, stream=None):
        """CR-(RC)^n front-end shaping of Eq. 1 currents (device tensors)."""
        return B.wt_shape(self.ctx, i, dt, tau, order, gain, noise, noise_rms, out, stream)

    def tuning(self):
        """Launch shapes of the FP32 path (nb, lb, nch, nepi), set by the autotuner."""
        return B.wt_get_tuning(self.ctx)

    def sync(self, stream=None):
        """Wait and raise on a device-side failure of earlier asynchronous calls."""
        B.wt_sync(self.ctx, stream)

    def charges(self):
        return B.wt_get_charges(self.ctx, len(self.times), self.n_sources)

    def capacitance(self):
        return B.wt_get_capacitance(self.ctx, self.n_sources)

    def modes(self):
        return B.wt_get_modes(self.ctx, self.n_sources)

    def info(self):
        return B.wt_get_info(self.ctx)

    def set_timing(self, enable=True):
        B.wt_set_timing(self.ctx, enable)

    def timing(self):
        return B.wt_get_timing(self.ctx)

    def grad_timing(self):
        return B.wt_get_grad_timing(self.ctx)

    def close(self):
        if self.ctx:
            B.wt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
