"""Band-limited periodic fundamental solution of the Poisson operator.

Reading of the Abstract ("fundamental solutions to impose boundary conditions
and spectral methods to extend the solution to the bulk") and Sec. 3 (spectra
multiplied or divided by the squared wave-vector |k|^2):

    g(d) = 1/(eps V') * sum_{k != 0} exp(i k.d) / |k|^2

over the band-limited mode set of the voxel grid (Nyquist modes dropped, so
every field is a real trigonometric polynomial; the k = 0 term is dropped,
i.e. a neutralising background, exact for the neutral charge sets used here).

Lateral (x, y): periodic with periods Lx, Ly, modes k = 2 pi m / L,
|m| <= N/2 - 1.  Vertical (z): "mirror" (default) reflects the sensor at
z = 0 and z = Lz (Neumann), realised as a periodic box of height 2 Lz with an
image charge at -z_s, modes k_z = pi m / Lz, |m| <= Nz - 1; V' = Lx Ly 2 Lz.
"periodic" uses k_z = 2 pi m / Lz, |m| <= Nz/2 - 1 and V' = Lx Ly Lz.

``ewald_green`` is an independent Ewald lattice sum of the exact (not band-
limited) periodic Green's function with the same neutralising background.  It
is used only to pin ``green_direct``.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

EPS0 = 8.8541878128e-12


def eps_abs(grid) -> float:
    return EPS0 * grid.eps_r


def mode_sets(grid):
    """Symmetric mode sets (kx, ky, kz) and the periodic volume V'."""
    for n in (grid.Nx, grid.Ny):
        if n % 2:
            raise ValueError("Nx and Ny must be even")
    mx = np.arange(-(grid.Nx // 2 - 1), grid.Nx // 2)
    my = np.arange(-(grid.Ny // 2 - 1), grid.Ny // 2)
    kx = 2.0 * math.pi * mx / grid.Lx
    ky = 2.0 * math.pi * my / grid.Ly
    if grid.zbc == "mirror":
        mz = np.arange(-(grid.Nz - 1), grid.Nz)
        kz = math.pi * mz / grid.Lz
        vol = grid.Lx * grid.Ly * 2.0 * grid.Lz
    elif grid.zbc == "periodic":
        if grid.Nz % 2:
            raise ValueError("Nz must be even for periodic z")
        mz = np.arange(-(grid.Nz // 2 - 1), grid.Nz // 2)
        kz = 2.0 * math.pi * mz / grid.Lz
        vol = grid.Lx * grid.Ly * grid.Lz
    else:
        raise ValueError(grid.zbc)
    return kx, ky, kz, vol


def inv_k2(kx, ky, kz):
    """1/|k|^2 on the full tensor mode grid, 0 at k = 0."""
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    with np.errstate(divide="ignore"):
        out = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    return out


def green_direct(grid, d):
    """g(d) for offsets d [n, 3] by the plain sum over every mode (small grids)."""
    kx, ky, kz, vol = mode_sets(grid)
    ik2 = inv_k2(kx, ky, kz)
    d = np.atleast_2d(np.asarray(d, dtype=float))
    out = np.empty(len(d))
    for i, (dx, dy, dz) in enumerate(d):
        ph = (np.exp(1j * kx * dx)[:, None, None] * np.exp(1j * ky * dy)[None, :, None]
              * np.exp(1j * kz * dz)[None, None, :])
        out[i] = np.real(np.sum(ph * ik2))
    return out / (eps_abs(grid) * vol)


def unit_potential_direct(grid, targets, sources):
    """Phi[i, j]: potential at targets[i] from a unit point source at sources[j]
    (plus its mirror image at -z for the mirror boundary), by green_direct."""
    targets = np.atleast_2d(targets)
    sources = np.atleast_2d(sources)
    out = np.empty((len(targets), len(sources)))
    for j, s in enumerate(sources):
        out[:, j] = green_direct(grid, targets - s)
        if grid.zbc == "mirror":
            out[:, j] += green_direct(grid, targets - s * np.array([1.0, 1.0, -1.0]))
    return out


def _lateral_groups(p):
    """Unique lateral (x, y) positions and the group index of each point."""
    uniq, inv = np.unique(np.asarray(p)[:, :2], axis=0, return_inverse=True)
    return uniq, inv.ravel()


def lateral_table(grid, dxy, kz_half):
    """L[c, m] = sum over lateral modes of cos(kx dx + ky dy) / |k|^2 at k_z =
    kz_half[m] (k = 0 excluded), for each lateral offset dxy[c]."""
    kx, ky, _, _ = mode_sets(grid)
    ik2 = inv_k2(kx, ky, kz_half)                      # [nkx, nky, nkz]
    out = np.empty((len(dxy), len(kz_half)))
    for c, (dx, dy) in enumerate(dxy):
        ex = np.exp(1j * kx * dx)
        ey = np.exp(1j * ky * dy)
        t = np.tensordot(ex, ik2, axes=(0, 0))          # [nky, nkz]
        out[c] = np.real(np.tensordot(ey, t, axes=(0, 0)))
    return out


def potential_matrix(grid, targets, sources):
    """Phi[i, j] for many targets and sources that share few lateral positions
    (points on column axes and column surfaces).  Same sum as
    unit_potential_direct, evaluated per (target lateral position, source
    lateral position) pair: the lateral part of the mode sum first, then the
    z part as a product of cosine tables."""
    targets = np.asarray(targets, dtype=float)
    sources = np.asarray(sources, dtype=float)
    _, _, kz, vol = mode_sets(grid)
    tu, tinv = _lateral_groups(targets)
    su, sinv = _lateral_groups(sources)
    if grid.zbc == "mirror":
        kzh = kz[kz >= 0]                                  # 0 .. (Nz-1) pi / Lz
        w = np.where(kzh > 0, 2.0, 1.0)                    # +-kz pairs
    else:
        kzh = kz[kz >= 0]
        w = np.where(kzh > 0, 2.0, 1.0)
    dxy = (tu[:, None, :] - su[None, :, :]).reshape(-1, 2)
    L = lateral_table(grid, dxy, kzh).reshape(len(tu), len(su), len(kzh))
    pref = 1.0 / (eps_abs(grid) * vol)
    out = np.empty((len(targets), len(sources)))
    for a in range(len(tu)):
        ti = np.nonzero(tinv == a)[0]
        ct = np.cos(np.outer(targets[ti, 2], kzh))
        st = np.sin(np.outer(targets[ti, 2], kzh))
        for b in range(len(su)):
            sj = np.nonzero(sinv == b)[0]
            cs = np.cos(np.outer(sources[sj, 2], kzh))
            coef = w * L[a, b]
            if grid.zbc == "mirror":
                # source + image: exp(ikz(zt-zs)) + exp(ikz(zt+zs)) summed over +-kz
                blk = 2.0 * (ct * coef) @ cs.T
            else:
                ss = np.sin(np.outer(sources[sj, 2], kzh))
                blk = (ct * coef) @ cs.T + (st * coef) @ ss.T
            out[np.ix_(ti, sj)] = pref * blk
    return out


def ewald_green(box, d, eps, alpha=None, n_real=4, k_cut=None):
    """Exact periodic Green's function of a unit point charge with a uniform
    neutralising background (zero cell average), by Ewald summation:

        g = 1/(4 pi eps) sum_n erfc(a |d+n|)/|d+n|
          + 1/(eps V) sum_{k != 0} exp(-k^2/(4 a^2)) exp(i k.d)/k^2
          - 1/(4 eps a^2 V)

    ``box`` = (Lx, Ly, Lz) periods.  Independent of the band-limited sum."""
    box = np.asarray(box, dtype=float)
    d = np.atleast_2d(np.asarray(d, dtype=float))
    vol = float(np.prod(box))
    if alpha is None:
        alpha = 5.0 / box.min()
    rng = np.arange(-n_real, n_real + 1)
    shifts = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) * box
    out = np.zeros(len(d))
    for i, di in enumerate(d):
        r = np.linalg.norm(di[None, :] + shifts, axis=1)
        out[i] = np.sum(erfc(alpha * r) / r) / (4.0 * math.pi * eps)
    if k_cut is None:
        k_cut = 2.0 * alpha * 6.5
    ms = [np.arange(-int(k_cut * L / (2 * math.pi)) - 1, int(k_cut * L / (2 * math.pi)) + 2) for L in box]
    kx = 2 * math.pi * ms[0] / box[0]
    ky = 2 * math.pi * ms[1] / box[1]
    kz = 2 * math.pi * ms[2] / box[2]
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        wk = np.where(k2 > 0, np.exp(-k2 / (4 * alpha * alpha)) / np.where(k2 > 0, k2, 1.0), 0.0)
    for i, (dx, dy, dz) in enumerate(d):
        ph = (np.exp(1j * kx * dx)[:, None, None] * np.exp(1j * ky * dy)[None, :, None]
              * np.exp(1j * kz * dz)[None, None, :])
        out[i] += np.real(np.sum(wk * ph)) / (eps * vol)
    out -= 1.0 / (4.0 * eps * alpha * alpha * vol)
    return out
