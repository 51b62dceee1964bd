"""Pseudo-spectral extension of the weighting potential and field into the
bulk at each time sample (Abstract: spectral methods extend the solution to
the bulk; Sec. 1: discrete Fourier transforms; Sec. 3: spectra divided by
|k|^2).

With node charges q_j(t) at source positions s_j,

    rho^(k, t) = sum_j q_j(t) exp(-i k_perp . s_perp_j) Z(k_z, s_zj)
        Z = 2 cos(k_z s_z)  (mirror: source plus image)  or exp(-i k_z s_z),
    psi(x, t)  = 1/(eps V') Re sum_{k != 0} rho^ exp(i k.x) / |k|^2,
    W_a(x, t)  = -d psi / d x_a = 1/(eps V') Re sum_k (-i k_a) rho^ exp(i k.x) / |k|^2.

W = -grad psi is the field the library stores as H (3 components, V/m);
grid points are x_i = i Lx/Nx, y_j = j Ly/Ny, z_k = (k + 1/2) Lz/Nz.  The
sums are evaluated directly: separable per axis on tensor-product point sets,
mode by mode at scattered points.  No FFT is used.
"""
from __future__ import annotations

import numpy as np

from .greens import mode_sets, inv_k2, eps_abs


def grid_coords(grid):
    x = np.arange(grid.Nx) * grid.Lx / grid.Nx
    y = np.arange(grid.Ny) * grid.Ly / grid.Ny
    z = (np.arange(grid.Nz) + 0.5) * grid.Lz / grid.Nz
    return x, y, z


def _zfactor(grid, kz, sz):
    if grid.zbc == "mirror":
        return 2.0 * np.cos(np.outer(kz, sz))
    return np.exp(-1j * np.outer(kz, sz))


def rho_hat(grid, src, q):
    """rho^[t, mx, my, mz] for charges q [Ns, nt] (one time: q [Ns])."""
    q = np.asarray(q, dtype=float)
    if q.ndim == 1:
        q = q[:, None]
    kx, ky, kz, _ = mode_sets(grid)
    uniq, inv = np.unique(src[:, :2], axis=0, return_inverse=True)
    inv = inv.ravel()
    zf = _zfactor(grid, kz, src[:, 2])                      # [nkz, Ns]
    out = np.zeros((q.shape[1], len(kx), len(ky), len(kz)), dtype=complex)
    for u, (xu, yu) in enumerate(uniq):
        sel = inv == u
        Zu = zf[:, sel] @ q[sel]                             # [nkz, nt]
        lat = np.exp(-1j * kx * xu)[:, None] * np.exp(-1j * ky * yu)[None, :]
        out += lat[None, :, :, None] * Zu.T[:, None, None, :]
    return out


def _spectral_factor(grid, rh, comp):
    """Per-mode factor of component comp: 0,1,2 = field x,y,z; 3 = potential."""
    kx, ky, kz, vol = mode_sets(grid)
    f = rh * inv_k2(kx, ky, kz)
    if comp == 0:
        f = f * (-1j * kx)[:, None, None]
    elif comp == 1:
        f = f * (-1j * ky)[None, :, None]
    elif comp == 2:
        f = f * (-1j * kz)[None, None, :]
    return f / (eps_abs(grid) * vol)


def field_subgrid(grid, src, q, ix=None, iy=None, iz=None, comps=(0, 1, 2)):
    """W[t, comp, i, j, k] on the tensor-product subgrid of grid indices
    ix x iy x iz (None = all).  comp 3 is the potential psi."""
    kx, ky, kz, _ = mode_sets(grid)
    x, y, z = grid_coords(grid)
    ix = np.arange(grid.Nx) if ix is None else np.asarray(ix)
    iy = np.arange(grid.Ny) if iy is None else np.asarray(iy)
    iz = np.arange(grid.Nz) if iz is None else np.asarray(iz)
    ex = np.exp(1j * np.outer(kx, x[ix]))
    ey = np.exp(1j * np.outer(ky, y[iy]))
    ez = np.exp(1j * np.outer(kz, z[iz]))
    q = np.asarray(q, dtype=float)
    if q.ndim == 1:
        q = q[:, None]
    out = np.empty((q.shape[1], len(comps), len(ix), len(iy), len(iz)))
    for t in range(q.shape[1]):
        rh = rho_hat(grid, src, q[:, t])[0]
        for ci, c in enumerate(comps):
            f = _spectral_factor(grid, rh, c)
            g = np.tensordot(f, ez, axes=(2, 0))             # [mx, my, k]
            g = np.tensordot(g, ey, axes=(1, 0))             # [mx, k, j]
            g = np.tensordot(g, ex, axes=(0, 0))             # [k, j, i]
            out[t, ci] = np.real(g).transpose(2, 1, 0)
    return out


def field_points(grid, src, q, pts, comps=(0, 1, 2)):
    """W[t, n, comp] at scattered points pts [n, 3], mode by mode."""
    kx, ky, kz, _ = mode_sets(grid)
    pts = np.atleast_2d(np.asarray(pts, dtype=float))
    q = np.asarray(q, dtype=float)
    if q.ndim == 1:
        q = q[:, None]
    out = np.empty((q.shape[1], len(pts), len(comps)))
    for t in range(q.shape[1]):
        rh = rho_hat(grid, src, q[:, t])[0]
        fs = [_spectral_factor(grid, rh, c) for c in comps]
        for n, (px, py, pz) in enumerate(pts):
            ph = (np.exp(1j * kx * px)[:, None, None] * np.exp(1j * ky * py)[None, :, None]
                  * np.exp(1j * kz * pz)[None, None, :])
            for ci, f in enumerate(fs):
                out[t, n, ci] = np.real(np.sum(f * ph))
    return out
