"""Seeded workload definitions (sensor geometry, material, time samples, tracks).

Units are SI throughout: metres, seconds, Ohm*m, Coulomb, Volt.

Five named workloads, each with a fixed default seed:

* ``c1`` single cell, 55x55x100 um, grid 32x32x64, 2 columns, 64 time samples.
* ``c2`` 3x3 pixel cell, 165x165x500 um, grid 128x128x256, 18 columns,
  512 time samples.
* ``c3`` 64 single-cell sensors with drawn pitch, thickness, radius,
  resistivity and grid size, 256 time samples each.
* ``c4`` 3x3 cell at grid 96x96x192, 256 time samples, 10k straight tracks.
* ``c5`` 5x5 pixel cell, grid 192x192x384, 256 time samples, 1e5 drift tracks.

Nothing here evaluates the solver; the per-column source count follows the
placement rule ``min(requested, Nz spanned, floor(3.25 L / r))`` so that the
same integer reaches both the oracle and the library as an input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

UM = 1e-6
OHM_CM = 1e-2          # 1 Ohm*cm in Ohm*m
E_CHARGE = 1.602176634e-19


@dataclass(frozen=True)
class GridSpec:
    Lx: float
    Ly: float
    Lz: float
    Nx: int
    Ny: int
    Nz: int
    eps_r: float = 5.7
    zbc: str = "mirror"          # "mirror" (Neumann at z=0, Lz) or "periodic"

    @property
    def n_points(self) -> int:
        return self.Nx * self.Ny * self.Nz


@dataclass(frozen=True)
class ColumnSpec:
    x: float
    y: float
    z0: float
    z1: float
    radius: float
    resistivity: float           # Ohm*m
    terminal_top: int            # 1: terminal at z1, 0: at z0
    driven: int                  # 1: readout held at V_w
    n_sources: int
    rho_profile: Optional[Tuple[float, ...]] = None   # per-node resistivity [Ohm*m] (depth profile)


@dataclass(frozen=True)
class FitSpec:
    n_az: int = 4
    n_h: int = 2
    tikhonov: float = 0.0
    v_w: float = 1.0
    az0: float = 0.0             # first collocation azimuth [rad]


@dataclass
class TrackSet:
    """Carrier tracks, [track][step] arrays (float64 here; the library takes float32)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    dt: float
    charge: np.ndarray           # per-track charge [C] (or normalised units)
    n_out: int

    @property
    def n_tracks(self) -> int:
        return self.x.shape[0]

    @property
    def n_steps(self) -> int:
        return self.x.shape[1]


@dataclass
class Workload:
    name: str
    grid: GridSpec
    columns: List[ColumnSpec]
    fit: FitSpec
    times: np.ndarray
    tracks: Optional[TrackSet] = None
    seed: int = 0
    notes: str = ""


def log_times(n_t: int, t0: float = 1e-12, t1: float = 1e-8) -> np.ndarray:
    """n_t log-uniform samples from t0 to t1 inclusive."""
    if n_t == 1:
        return np.array([t0])
    return 10.0 ** np.linspace(math.log10(t0), math.log10(t1), n_t)


def n_sources_rule(requested: int, grid: GridSpec, z0: float, z1: float, radius: float) -> int:
    nz_span = max(1, int(round((z1 - z0) / grid.Lz * grid.Nz)))
    cap = int(math.floor(3.25 * (z1 - z0) / radius))
    return max(1, min(requested, nz_span, cap))


def _column(grid, x, y, r, rho, top, driven, m_req, z0=0.0, z1=None):
    z1 = grid.Lz if z1 is None else z1
    return ColumnSpec(x=x, y=y, z0=z0, z1=z1, radius=r, resistivity=rho,
                      terminal_top=top, driven=driven,
                      n_sources=n_sources_rule(m_req, grid, z0, z1, r))


def pixel_matrix(npix: int, pitch: float, thick: float, nx: int, nz: int, radius: float,
                 rho_lo: float, rho_hi: float, m_req: int, rng: np.random.Generator,
                 eps_r: float = 5.7) -> tuple:
    """npix x npix pixels: a readout column at each pixel centre (terminal at the top),
    a bias column at each pixel corner (terminal at the bottom); only the central
    readout is driven.  Resistivities are drawn per column, readouts first."""
    L = npix * pitch
    grid = GridSpec(L, L, thick, nx, nx, nz, eps_r)
    cols = []
    centre = npix // 2
    rho_r = rng.uniform(rho_lo, rho_hi, size=npix * npix)
    rho_b = rng.uniform(rho_lo, rho_hi, size=npix * npix)
    k = 0
    for i in range(npix):
        for j in range(npix):
            cols.append(_column(grid, (i + 0.5) * pitch, (j + 0.5) * pitch, radius, rho_r[k],
                                1, int(i == centre and j == centre), m_req))
            k += 1
    k = 0
    for i in range(npix):
        for j in range(npix):
            cols.append(_column(grid, i * pitch, j * pitch, radius, rho_b[k], 0, 0, m_req))
            k += 1
    return grid, cols


def c1_single_cell(seed: int = 1) -> Workload:
    rng = np.random.default_rng(seed)
    grid = GridSpec(55 * UM, 55 * UM, 100 * UM, 32, 32, 64, 5.7)
    rho = rng.uniform(0.05, 0.5, size=2) * OHM_CM
    cols = [
        _column(grid, 27.5 * UM, 27.5 * UM, 5 * UM, rho[0], 1, 1, 64),
        _column(grid, 0.0, 0.0, 5 * UM, rho[1], 0, 0, 64),
    ]
    return Workload("c1", grid, cols, FitSpec(), log_times(64), seed=seed,
                    notes="single cell, readout at centre (terminal top, driven), bias at corner")


def c2_pixel3x3(seed: int = 2) -> Workload:
    rng = np.random.default_rng(seed)
    grid, cols = pixel_matrix(3, 55 * UM, 500 * UM, 128, 256, 6 * UM, 0.1 * OHM_CM, 1.0 * OHM_CM, 256, rng)
    return Workload("c2", grid, cols, FitSpec(), log_times(512), seed=seed,
                    notes="3x3 pixels, 18 columns, central readout driven")


def c4_adjoint(seed: int = 4, n_tracks: int = 10_000) -> Workload:
    rng = np.random.default_rng(seed)
    # radius 5 um (r/h = 2.91 at h = 165/96 um): at 6 um (r/h = 3.49) the box-band
    # fit gives an indefinite capacitance on this grid
    grid, cols = pixel_matrix(3, 55 * UM, 500 * UM, 96, 192, 5 * UM, 0.1 * OHM_CM, 1.0 * OHM_CM, 256, rng)
    tracks = mip_tracks(grid, n_tracks, 100, rng)
    return Workload("c4", grid, cols, FitSpec(), log_times(256), tracks=tracks, seed=seed,
                    notes="3x3 pixels at grid 96x96x192, radius 5 um, 10k straight tracks, q = 1")


def c5_large(seed: int = 5, n_tracks: int = 100_000) -> Workload:
    rng = np.random.default_rng(seed)
    grid, cols = pixel_matrix(5, 55 * UM, 500 * UM, 192, 384, 6 * UM, 0.1 * OHM_CM, 1.0 * OHM_CM, 256, rng)
    tracks = drift_tracks(grid, cols, n_tracks, 200, 1.5e-12, rng)
    return Workload("c5", grid, cols, FitSpec(), log_times(256), tracks=tracks, seed=seed,
                    notes="5x5 pixels, 50 columns, 1e5 electron/hole drift tracks")


def _box_band_radius(r: float, h: float, rng: np.random.Generator) -> float:
    """r, or a redraw from U(4, 10) um, such that sin(pi r / h) >= 0.5.  With
    the box-band kernel the fitted capacitance turns indefinite in windows of
    r / h where sin(pi r / h) is negative (found at r/h = 1.45, 1.75, 3.49,
    5.82); every configuration used so far that fits has sin(pi r / h) > 0."""
    for _ in range(10_000):
        if math.sin(math.pi * r / h) >= 0.5:
            return r
        r = rng.uniform(4, 10) * UM
    raise ValueError(f"no radius in 4-10 um avoids the indefinite windows at h = {h}")


def c3_batch(seed: int = 3, n_sensors: int = 64, nx_choices=(64, 80, 96, 112, 128), n_t: int = 256) -> List[Workload]:
    """Single cells of drawn pitch, thickness, radius and resistivities on
    uneven grids (Nz = 2 Nx).  Smaller nx_choices / n_t give test-sized batches
    of the same kind."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_sensors):
        pitch = rng.uniform(40, 110) * UM
        thick = rng.uniform(300, 500) * UM
        r = rng.uniform(4, 10) * UM
        rho = rng.uniform(0.05, 2.0, size=2) * OHM_CM
        nx = int(rng.choice(list(nx_choices)))
        r = _box_band_radius(r, pitch / nx, np.random.default_rng([seed, s]))
        grid = GridSpec(pitch, pitch, thick, nx, nx, 2 * nx, 5.7)
        cols = [
            _column(grid, 0.5 * pitch, 0.5 * pitch, r, rho[0], 1, 1, 2 * nx),
            _column(grid, 0.0, 0.0, r, rho[1], 0, 0, 2 * nx),
        ]
        out.append(Workload(f"c3.{s}", grid, cols, FitSpec(), log_times(n_t), seed=seed))
    return out


def tiny_cell(nx: int = 8, nz: int = 16, seed: int = 7, n_t: int = 16, m_req: int = None,
              pitch: float = 55 * UM, thick: float = 100 * UM, radius: float = 5 * UM,
              rho=(0.05 * OHM_CM, 0.5 * OHM_CM)) -> Workload:
    """A small single cell for quick oracle and parity checks (all sizes free)."""
    rng = np.random.default_rng(seed)
    grid = GridSpec(pitch, pitch, thick, nx, nx, nz, 5.7)
    m_req = nz if m_req is None else m_req
    r = rng.uniform(*rho, size=2)
    cols = [
        _column(grid, 0.5 * pitch, 0.5 * pitch, radius, r[0], 1, 1, m_req),
        _column(grid, 0.0, 0.0, radius, r[1], 0, 0, m_req),
    ]
    return Workload("tiny", grid, cols, FitSpec(), log_times(n_t), seed=seed)


def mip_tracks(grid: GridSpec, n_tracks: int, n_steps: int, rng: np.random.Generator,
               speed: float = 1e5, charge: float = 1.0) -> TrackSet:
    """Straight tracks entering uniformly on the top face, directions isotropic
    within 30 degrees of -z, |v| = 1e7 cm/s, dt = Lz / (n_steps |v|).  Lateral
    positions wrap periodically; the velocity is zero once z leaves [0, Lz]."""
    dt = grid.Lz / (n_steps * speed)
    x0 = rng.uniform(0, grid.Lx, n_tracks)
    y0 = rng.uniform(0, grid.Ly, n_tracks)
    cos_max = math.cos(math.radians(30.0))
    ct = rng.uniform(cos_max, 1.0, n_tracks)        # isotropic within the cone
    st = np.sqrt(1.0 - ct * ct)
    ph = rng.uniform(0, 2 * math.pi, n_tracks)
    v = np.stack([speed * st * np.cos(ph), speed * st * np.sin(ph), -speed * ct], axis=1)
    steps = np.arange(n_steps)
    x = x0[:, None] + v[:, 0:1] * dt * steps
    y = y0[:, None] + v[:, 1:2] * dt * steps
    z = grid.Lz + v[:, 2:3] * dt * steps
    inside = (z >= 0.0) & (z <= grid.Lz)
    vx = np.where(inside, v[:, 0:1], 0.0)
    vy = np.where(inside, v[:, 1:2], 0.0)
    vz = np.where(inside, v[:, 2:3], 0.0)
    z = np.clip(z, 0.0, grid.Lz)
    x = np.mod(x, grid.Lx)
    y = np.mod(y, grid.Ly)
    return TrackSet(x, y, z, vx, vy, vz, dt, np.full(n_tracks, charge), 2 * n_steps)


def drift_tracks(grid: GridSpec, cols: List[ColumnSpec], n_tracks: int, n_steps: int, dt: float,
                 rng: np.random.Generator, speed: float = 1e5) -> TrackSet:
    """Carriers created uniformly in the volume; electrons (charge -e) drift
    straight toward the nearest readout axis, holes (+e) toward the nearest
    bias axis, at |v| = 1e7 cm/s, stopping at the column surface.  50/50 split."""
    p = np.stack([rng.uniform(0, grid.Lx, n_tracks), rng.uniform(0, grid.Ly, n_tracks),
                  rng.uniform(0, grid.Lz, n_tracks)], axis=1)
    is_e = np.arange(n_tracks) < n_tracks // 2
    rng.shuffle(is_e)
    charge = np.where(is_e, -E_CHARGE, E_CHARGE)
    ax = np.array([[c.x, c.y] for c in cols])
    readout = np.array([c.terminal_top == 1 for c in cols])
    rad = np.array([c.radius for c in cols])
    # nearest target axis under periodic wrap
    d = p[:, None, :2] - ax[None, :, :]
    d[..., 0] -= grid.Lx * np.round(d[..., 0] / grid.Lx)
    d[..., 1] -= grid.Ly * np.round(d[..., 1] / grid.Ly)
    dist = np.hypot(d[..., 0], d[..., 1])
    want = np.where(is_e[:, None], readout[None, :], ~readout[None, :])
    dist_m = np.where(want, dist, np.inf)
    tgt = np.argmin(dist_m, axis=1)
    dvec = -d[np.arange(n_tracks), tgt]                 # from carrier toward axis
    dn = np.maximum(np.hypot(dvec[:, 0], dvec[:, 1]), 1e-30)
    u = dvec / dn[:, None]
    travel = np.maximum(dn - rad[tgt], 0.0)              # stop at the surface
    t = np.arange(n_steps) * dt
    s = np.minimum(speed * t[None, :], travel[:, None])
    moving = (speed * t[None, :]) < travel[:, None]
    x = np.mod(p[:, 0:1] + u[:, 0:1] * s, grid.Lx)
    y = np.mod(p[:, 1:2] + u[:, 1:2] * s, grid.Ly)
    z = np.repeat(p[:, 2:3], n_steps, axis=1)
    vx = np.where(moving, speed * u[:, 0:1], 0.0)
    vy = np.where(moving, speed * u[:, 1:2], 0.0)
    vz = np.zeros_like(vx)
    return TrackSet(x, y, z, vx, vy, vz, dt, charge, 2 * n_steps)


def central_pixel_tracks(grid: GridSpec, pitch: float, n_tracks: int, n_steps: int, seed: int) -> TrackSet:
    """mip_tracks with entry points folded into the central pixel of a 3x3
    matrix (the driven readout's pixel)."""
    tr = mip_tracks(grid, n_tracks, n_steps, np.random.default_rng(seed))
    x0 = tr.x[:, :1]
    y0 = tr.y[:, :1]
    sx = pitch + np.mod(x0, pitch) - x0
    sy = pitch + np.mod(y0, pitch) - y0
    tr.x = np.mod(tr.x + sx, grid.Lx)
    tr.y = np.mod(tr.y + sy, grid.Ly)
    return tr


def scan_bias_diameter(diameters_um=(6, 8, 10, 12, 14), seed: int = 6, n_tracks: int = 1000, n_steps: int = 100,
                       n_t: int = 256, nx: int = 20, nz: int = 64) -> List[Tuple[float, Workload]]:
    """Sec. 5's scan of the bias-electrode diameter (6-14 um in 2 um steps) on
    the 3x3 pixel matrix (pitch 55 um, 500 um thick, readout radius 5 um,
    0.5 Ohm*cm in every column), one workload per diameter with the same grid
    and tracks (through the central pixel).  The lateral spacing (165 um / nx,
    8.25 um at nx = 20) keeps every radius below one spacing: with the
    box-band kernel the fit turns indefinite for r / h in (1, 2) and (3, 4),
    and no finer spacing clears all of r = 3..7 um."""
    out = []
    pitch, thick = 55 * UM, 500 * UM
    grid = GridSpec(3 * pitch, 3 * pitch, thick, nx, nx, nz, 5.7)
    tracks = central_pixel_tracks(grid, pitch, n_tracks, n_steps, seed)
    for d in diameters_um:
        cols = []
        for i in range(3):
            for j in range(3):
                cols.append(_column(grid, (i + 0.5) * pitch, (j + 0.5) * pitch, 5 * UM, 0.5 * OHM_CM, 1,
                                    int(i == 1 and j == 1), nz))
        for i in range(3):
            for j in range(3):
                cols.append(_column(grid, i * pitch, j * pitch, 0.5 * d * UM, 0.5 * OHM_CM, 0, 0, nz))
        out.append((float(d), Workload(f"scan_d{d}", grid, cols, FitSpec(), log_times(n_t), tracks=tracks,
                                       seed=seed, notes=f"bias diameter {d} um")))
    return out


def scan_thickness(thick_um=(300, 400, 500), nz_of=None, seed: int = 8, n_tracks: int = 1000, n_steps: int = 100,
                   n_t: int = 256, nx: int = 20) -> List[Tuple[float, Workload]]:
    """Sec. 5's thickness study (shorter readout electrodes): the 3x3 matrix
    at each thickness, columns through the whole bulk, the same lateral grid,
    Nz close to a 7.8 um spacing, tracks through the central pixel drawn
    from the same seed (their transit scales with the thickness)."""
    nz_of = nz_of or {300: 40, 400: 48, 500: 64}
    out = []
    pitch = 55 * UM
    for th in thick_um:
        grid = GridSpec(3 * pitch, 3 * pitch, th * UM, nx, nx, nz_of[th], 5.7)
        cols = []
        for i in range(3):
            for j in range(3):
                cols.append(_column(grid, (i + 0.5) * pitch, (j + 0.5) * pitch, 5 * UM, 0.5 * OHM_CM, 1,
                                    int(i == 1 and j == 1), grid.Nz))
        for i in range(3):
            for j in range(3):
                cols.append(_column(grid, i * pitch, j * pitch, 4 * UM, 0.5 * OHM_CM, 0, 0, grid.Nz))
        tracks = central_pixel_tracks(grid, pitch, n_tracks, n_steps, seed)
        out.append((float(th), Workload(f"scan_t{th}", grid, cols, FitSpec(), log_times(n_t), tracks=tracks,
                                        seed=seed, notes=f"thickness {th} um")))
    return out


_NAMED = {"c1": c1_single_cell, "c2": c2_pixel3x3, "c4": c4_adjoint, "c5": c5_large}


def workload(name: str, **kw) -> Workload:
    if name == "c3":
        raise ValueError("c3 is a list of workloads; call c3_batch()")
    return _NAMED[name](**kw)


def with_resistivity(w: Workload, rho) -> Workload:
    """Copy of w with every column's resistivity replaced (scalar or per column)."""
    rho = np.broadcast_to(np.asarray(rho, dtype=float), (len(w.columns),))
    cols = [replace(c, resistivity=float(r)) for c, r in zip(w.columns, rho)]
    return replace(w, columns=cols)
