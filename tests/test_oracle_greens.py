"""Pins of the oracle's fundamental solution (greens.py)."""
import math

import numpy as np
import pytest

from oracle import greens as G
from workloads.configs import GridSpec
from tests.golden.read import values

EPS = G.EPS0 * 5.7


def test_ewald_simple_cubic_constant():
    xi = values("ewald_simple_cubic.txt")["xi"]
    L = 1.0
    for r in (1e-3, 1e-2):
        g = G.ewald_green((L, L, L), [[r, 0.0, 0.0]], EPS)[0]
        lhs = (g - 1.0 / (4 * math.pi * EPS * r)) * 4 * math.pi * EPS * L
        assert abs(lhs - (xi + 2 * math.pi / 3 * r * r)) < 2e-5


def test_ewald_alpha_independent_and_zero_mean():
    box = (1.0, 1.3, 0.7)
    d = [[0.2, 0.1, 0.3], [0.45, -0.6, 0.05]]
    a = G.ewald_green(box, d, EPS, alpha=3.0)
    b = G.ewald_green(box, d, EPS, alpha=8.0)
    assert np.allclose(a, b, rtol=1e-12)
    # zero cell average: midpoint rule on a coarse lattice away from the charge
    n = 6
    u = (np.arange(n) + 0.5) / n
    pts = np.stack(np.meshgrid(u * box[0], u * box[1], u * box[2], indexing="ij"), -1).reshape(-1, 3)
    mean = G.ewald_green(box, pts + 1e-3, EPS).mean()
    scale = 1.0 / (4 * math.pi * EPS * min(box))
    assert abs(mean) < 0.05 * scale


@pytest.mark.parametrize("zbc", ["periodic", "mirror"])
def test_band_limited_green_converges_to_ewald(zbc):
    """g (band-limited) -> exact periodic Green's function as the grid refines."""
    L = 40e-6
    d = np.array([[9.3e-6, 4.1e-6, 6.7e-6], [15.0e-6, -11.0e-6, 3.0e-6]])
    box = (L, L, L if zbc == "periodic" else 2 * L)
    ref = G.ewald_green(box, d, EPS)
    errs = []
    for n in (8, 16, 32):
        grid = GridSpec(L, L, L, n, n, n if zbc == "periodic" else n // 2, 5.7, zbc)
        g = G.green_direct(grid, d)
        errs.append(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.05


def test_band_limited_green_near_field_is_coulomb():
    """h << r << L, off the lattice axes:
    g - 1/(4 pi eps r) -> xi/(4 pi eps L) + r^2/(6 eps V), error falling with N.
    (Along a lattice axis the box-shaped mode truncation leaves a Gibbs ridge
    that does not shrink with N, so this pin uses a generic direction.)"""
    xi = values("ewald_simple_cubic.txt")["xi"]
    L = 50e-6
    u = np.array([0.6, 0.48, 0.64])
    u /= np.linalg.norm(u)
    worst = []
    for n in (24, 48):
        grid = GridSpec(L, L, L, n, n, n, 5.7, "periodic")
        e = 0.0
        for r in (6e-6, 9e-6):
            g = G.green_direct(grid, [u * r])[0]
            model = 1 / (4 * math.pi * EPS * r) + xi / (4 * math.pi * EPS * L) + r * r / (6 * EPS * L ** 3)
            e = max(e, abs(g - model) / (1 / (4 * math.pi * EPS * r)))
        worst.append(e)
    assert worst[1] < worst[0]
    assert worst[1] < 5e-3


def test_green_symmetries():
    grid = GridSpec(30e-6, 40e-6, 50e-6, 8, 10, 12, 5.7, "mirror")
    d = np.array([[3e-6, 7e-6, 11e-6], [-5e-6, 2e-6, -4e-6]])
    assert np.allclose(G.green_direct(grid, d), G.green_direct(grid, -d), rtol=1e-13)
    # mirror: potential of source+image is even about z = 0 and z = Lz
    s = np.array([[4e-6, 9e-6, 13e-6]])
    t = np.array([[11e-6, 2e-6, 7e-6], [11e-6, 2e-6, -7e-6],
                  [11e-6, 2e-6, 50e-6 - 3e-6], [11e-6, 2e-6, 50e-6 + 3e-6]])
    phi = G.unit_potential_direct(grid, t, s)[:, 0]
    assert abs(phi[0] - phi[1]) < 1e-10 * abs(phi[0])
    assert abs(phi[2] - phi[3]) < 1e-10 * abs(phi[2])


@pytest.mark.parametrize("zbc", ["mirror", "periodic"])
def test_potential_matrix_matches_direct_sum(zbc):
    """The factorised evaluation used for the fit matrix equals the plain sum."""
    grid = GridSpec(30e-6, 36e-6, 40e-6, 8, 10, 12, 5.7, zbc)
    rng = np.random.default_rng(0)
    lat_t = rng.uniform(0, 30e-6, (3, 2))
    lat_s = rng.uniform(0, 30e-6, (2, 2))
    t = np.concatenate([np.c_[np.repeat(l[None], 4, 0), rng.uniform(0, 40e-6, 4)] for l in lat_t])
    s = np.concatenate([np.c_[np.repeat(l[None], 3, 0), rng.uniform(0, 40e-6, 3)] for l in lat_s])
    a = G.potential_matrix(grid, t, s)
    b = G.unit_potential_direct(grid, t, s)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-11 * np.abs(b).max())
